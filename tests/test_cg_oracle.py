"""Pins of the two-component colour-gradient oracle (paper section 2.1).

Checked against what the mathematics and the physics fix, not against the
oracle's own formulas: the single-colour limit is the single-component
oracle; each colour's mass and the total momentum are conserved; the
isotropic gradient of a sine equals its closed form; the perturbation weights
satisfy the two moment conditions of a mass-conserving capillary stress; and
a static droplet obeys Laplace's law dp = sigma / R in 2D with the input
surface tension.
"""
import math

import numpy as np
import pytest

import oracle
import synth

CS2 = 1.0 / 3.0


def _droplet(n, R, d=2, width=2.0):
    if d == 2:
        x, y = np.meshgrid(np.arange(n), np.arange(n), indexing="xy")
        r = np.sqrt((x - (n - 1) / 2) ** 2 + (y - (n - 1) / 2) ** 2).ravel()
    else:
        z, y, x = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
        r = np.sqrt((x - (n - 1) / 2) ** 2 + (y - (n - 1) / 2) ** 2 + (z - (n - 1) / 2) ** 2).ravel()
    phi = np.tanh((R - r) / width)
    return (1 + phi) / 2, (1 - phi) / 2


@pytest.mark.parametrize("lat", ["D2Q9", "D3Q19"])
def test_perturbation_weights_moment_conditions(lat):
    B = oracle.cg_weights(lat)
    c, w, _ = oracle.lattice_tables(lat)
    d = 2 if lat == "D2Q9" else 3
    assert abs(B.sum() - CS2) < 1e-15                    # mass: sum B = sum t (c.n)^2 = cs2
    assert np.abs(B @ c).max() < 1e-15
    M = np.einsum("a,ai,aj->ij", B, c[:, :d].astype(float), c[:, :d].astype(float))
    assert np.abs(M - CS2 * np.eye(d)).max() < 1e-15    # capillary stress ~ (n n - I)
    assert len(set(np.round(B, 15)[np.argsort((c * c).sum(1))])) <= 3  # depends on |c| only


@pytest.mark.parametrize("lat,dims", [("D2Q9", (24, 17, 1)), ("D3Q19", (10, 9, 8))])
def test_single_colour_limit_is_single_component_step(lat, dims):
    """rho_B = 0: phi = 1, no gradient, no perturbation, no recolouring --
    the step is the single-component regularized step."""
    d = 2 if lat == "D2Q9" else 3
    rho, u, pineq = synth.smooth_random_state(dims, d, seed=4)
    cfg1 = oracle.make_cfg(lat, dims, 0.83)
    f = oracle.init(cfg1, rho, u)
    cg = oracle.make_cg_cfg(lat, dims, 0.83, sigma=0.05, beta=0.7)
    fr, fb = f.copy(), np.zeros_like(f)
    fr2, fb2 = oracle.cg_run(cg, fr, fb, 5)
    ref = oracle.run(cfg1, f, 5)
    assert np.abs(fr2 - ref).max() < 1e-15 and not fb2.any()


@pytest.mark.parametrize("lat,dims", [("D2Q9", (40, 33, 1)), ("D3Q19", (16, 14, 12))])
def test_colour_masses_and_total_momentum_conserved(lat, dims):
    d = 2 if lat == "D2Q9" else 3
    n = dims[0]
    rr, rb = _droplet(n, n / 4, d) if dims[1] == n else (None, None)
    N = int(np.prod(dims))
    if rr is None:
        phi = np.tanh(np.sin(2 * math.pi * np.arange(N) / N * 3) * 3)
        rr, rb = (1 + phi) / 2, (1 - phi) / 2
    _, u, _ = synth.smooth_random_state(dims, d, seed=5)
    cfg = oracle.make_cg_cfg(lat, dims, 0.7, sigma=0.02, beta=0.6)
    fr, fb = oracle.cg_init(cfg, rr, rb, u)
    R0, B0, u0 = oracle.cg_fields(cfg, fr, fb)
    fr2, fb2 = oracle.cg_run(cfg, fr, fb, 100)
    R1, B1, u1 = oracle.cg_fields(cfg, fr2, fb2)
    assert abs(R1.sum() - R0.sum()) < 1e-12 * N
    assert abs(B1.sum() - B0.sum()) < 1e-12 * N
    assert np.abs(u1.sum(1) - u0.sum(1)).max() < 1e-13 * N


@pytest.mark.parametrize("lat,dims", [("D2Q9", (48, 6, 1)), ("D3Q19", (24, 5, 4))])
def test_isotropic_gradient_of_a_sine(lat, dims):
    """(1/cs2) sum_a t_a c_a phi(x + c_a) of phi = sin(kx) is sin(k) cos(kx)
    exactly on a periodic lattice (sum of t_a c_x^2 over c_x = 1 is 1/6)."""
    n = dims[0]
    k = 2 * math.pi * 3 / n
    x = np.arange(int(np.prod(dims))) % n
    phi = np.sin(k * x)
    cfg = oracle.make_cg_cfg(lat, dims, 0.8, 0.0, 0.0)
    grad = oracle.cg_gradient(cfg, phi)
    assert np.abs(grad[0] - math.sin(k) * np.cos(k * x)).max() < 1e-14
    assert np.abs(grad[1:]).max() < 1e-14


@pytest.mark.slow
def test_laplace_law_2d():
    """A static droplet in a periodic box: the pressure jump cs2 (rho_in -
    rho_out) times R equals the input surface tension (2D Laplace law) within
    5 %, and the agreement improves with R."""
    n, sigma = 64, 0.01
    ratios = []
    for R in (8, 12, 16):
        cfg = oracle.make_cg_cfg("D2Q9", (n, n), 1.0, sigma, 0.7)
        rr, rb = _droplet(n, R)
        fr, fb = oracle.cg_init(cfg, rr, rb)
        fr, fb = oracle.cg_run(cfg, fr, fb, 3000)
        Rr, Bb, u = oracle.cg_fields(cfg, fr, fb)
        rho = (Rr + Bb).reshape(n, n)
        c = n // 2
        dp = CS2 * (rho[c - 2:c + 2, c - 2:c + 2].mean() - rho[:4, :4].mean())
        ratios.append(dp * R / sigma)
        assert np.abs(u).max() < 1e-3  # only the small spurious currents of a static drop
    assert all(abs(r - 1) < 0.05 for r in ratios), ratios
    assert abs(ratios[-1] - 1) < abs(ratios[0] - 1)
