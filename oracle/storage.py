"""Storage rounding of the populations for the reduced-precision modes.

TEST INFRASTRUCTURE ONLY (part of the CPU oracle; see oracle/__init__.py).

The reduced-precision modes keep the arithmetic in full precision and store
each population shifted by its rest value, ft_a = f_a - t_a rho0, rounded to
the nearest value of a narrower binary format, ties to even.  The paper runs
in FP32 (section 4) and names lower precision as the way to relieve the
memory bound (sections 6 and 7); the shifted form is the reading this library
takes (the deviation ft is small, so the format's relative precision applies
to it rather than to f ~ t_a).

The formats are defined by their significand width p (including the leading
bit) and their smallest normal exponent emin:
    IEEE 754 binary16 ("FP16"):  p = 11, emin = -14 (subnormals below 2^-14)
    bfloat16 ("BF16"):           p = 8,  emin = -126 (the FP32 exponent range)
A value x with leading bit 2^E is a multiple of 2^(max(E, emin) - p + 1) in the
format; rounding to that quantum with round-half-even is the format's
round-to-nearest-even.  Overflow cannot occur for populations (|ft| < 1).
"""
from __future__ import annotations

import numpy as np

FORMATS = {"f16s": (11, -14), "bf16s": (8, -126)}


def quantum(x: np.ndarray, storage: str) -> np.ndarray:
    """Spacing of the storage format's values around x (its ulp)."""
    p, emin = FORMATS[storage]
    x = np.asarray(x, dtype=np.float64)
    _, e = np.frexp(x)  # x = m 2^e with 1/2 <= |m| < 1: leading bit 2^(e - 1)
    qexp = np.maximum(e - 1, emin) - (p - 1)
    return np.ldexp(np.ones_like(x), qexp)


def round_to_format(x: np.ndarray, storage: str) -> np.ndarray:
    """Round FP64 values to the nearest value of the storage format (ties to even)."""
    p, emin = FORMATS[storage]
    x = np.asarray(x, dtype=np.float64)
    _, e = np.frexp(x)
    qexp = np.maximum(e - 1, emin) - (p - 1)
    return np.ldexp(np.rint(np.ldexp(x, -qexp)), qexp)  # power-of-two scalings are exact


def round_populations(f: np.ndarray, weights: np.ndarray, storage: str, rho0: float = 1.0) -> np.ndarray:
    """The stored state of a reduced-precision mode: t_a rho0 + round(f_a - t_a rho0)."""
    if storage in ("f64",):
        return np.array(f, dtype=np.float64, copy=True)
    shift = (np.asarray(weights, dtype=np.float64) * rho0)[:, None]
    if storage == "f32":
        return shift + (f - shift).astype(np.float32).astype(np.float64)
    return shift + round_to_format(f - shift, storage)
