"""Pins of the two-component colour-gradient oracle (paper section 2.1).

Checked against what the mathematics and the physics fix, not against the
oracle's own formulas: the single-colour limit is the single-component
oracle; each colour's mass and the total momentum are conserved; the
isotropic gradient of a sine equals its closed form; the perturbation weights
satisfy the two moment conditions of a mass-conserving capillary stress; and
a static droplet obeys Laplace's law dp = sigma / R in 2D with the input
surface tension.  The near-contact interactions (section 2.2) are pinned by
flags worked out by hand on a film profile, by mirror symmetry, by the
momentum a body force must add, and by their effect: approaching droplets
coalesce without them and stay apart with them.
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


# ------------------------------------------------------------ near-contact
# interactions (paper section 2.2)

def _profile_field(ny=6):
    """A y-uniform D2Q9 phase field along x (periodic, 20 columns): droplets
    (+1) separated by films (-1) one, two and three nodes thick."""
    row = np.array([1, 1, 1, 1, 1, -1, 1, 1, 1, 1, -1, -1, 1, 1, 1, 1, 1, -1, -1, -1], float)
    return np.tile(row, ny), row.size, ny


@pytest.mark.parametrize("h,expected", [
    # h = 1: only the one-node film at x = 5 has non-bulk points on both
    # sides at distance 1 (x = 4 and 6); the two- and three-node films do not.
    (1, [4, 6]),
    # h = 2: bulk x = 5 -> {3, 7}; x = 10 -> {8, 12}; x = 11 -> {9, 13};
    # x = 18 -> {16, 0} (periodic); x = 17 and 19 see a bulk node at distance 2.
    (2, [0, 3, 7, 8, 9, 12, 13, 16]),
])
@pytest.mark.parametrize("lat", ["D2Q9", "D3Q19"])
def test_nci_flags_hand_worked_film_profile(h, expected, lat):
    """The flags of the section 2.2 test on a profile whose answer is worked
    out by hand: a bulk node (phi < -1 + eps) with non-bulk points at distance
    h along a pair of opposite directions flags those two points.  Diagonal
    directions give the same columns in a field uniform across x; the
    directions without an x component none (D2Q9: 6 rows; D3Q19: 5 x 4
    cross-sections)."""
    phi, nx, ny = _profile_field(6 if lat == "D2Q9" else 20)
    dims = (nx, ny) if lat == "D2Q9" else (nx, 5, 4)
    cfg = oracle.make_cg_cfg(lat, dims, 0.8, 0.01, 0.7, nci_amp=1e-3, nci_eps=0.1, nci_h=h)
    fl = oracle.cg_nci_flags(cfg, phi).reshape(-1, nx)
    assert (fl == fl[0]).all()
    assert list(np.nonzero(fl[0])[0]) == expected


def _two_spheres(n, R, gap, d=3, width=1.5, R2=None):
    R2 = R if R2 is None else R2
    if d == 3:
        z, y, x = np.meshgrid(np.arange(n), np.arange(n), np.arange(2 * n), indexing="ij")
        c = (n - 1) / 2
        r1 = np.sqrt((x - (n - gap / 2 - R)) ** 2 + (y - c) ** 2 + (z - c) ** 2)
        r2 = np.sqrt((x - (n + gap / 2 + R2)) ** 2 + (y - c) ** 2 + (z - c) ** 2)
    else:
        y, x = np.meshgrid(np.arange(n), np.arange(2 * n), indexing="ij")
        c = (n - 1) / 2
        r1 = np.sqrt((x - (n - gap / 2 - R)) ** 2 + (y - c) ** 2)
        r2 = np.sqrt((x - (n + gap / 2 + R2)) ** 2 + (y - c + 1.5) ** 2)
    return np.maximum(np.tanh((R - r1) / width), np.tanh((R2 - r2) / width)).ravel()


def test_nci_flags_d3q19_mirror_symmetric_in_the_gap():
    """Two equal spheres facing each other across a thin film: the flags are
    mirror symmetric about the mid-plane and all lie in the gap region."""
    n = 20
    phi = _two_spheres(n, 6.0, 3.0)
    cfg = oracle.make_cg_cfg("D3Q19", (2 * n, n, n), 0.8, 0.01, 0.7, nci_amp=1e-3, nci_eps=0.1, nci_h=2)
    fl = oracle.cg_nci_flags(cfg, phi).reshape(n, n, 2 * n)
    assert fl.sum() > 0
    x_mirror = (2 * n - np.arange(2 * n)) % (2 * n)  # mid-plane x = n (periodic box)
    assert np.array_equal(phi.reshape(n, n, 2 * n), phi.reshape(n, n, 2 * n)[:, :, x_mirror])
    assert np.array_equal(fl, fl[:, :, x_mirror])
    xs = np.nonzero(fl)[2]
    assert xs.min() >= n - 6 and xs.max() <= n + 6


def test_nci_off_or_without_films_is_plain_cg():
    """Amplitude 0, or a state with no film anywhere (one droplet), leaves
    the colour-gradient step exactly unchanged."""
    n = 40
    x, y = np.meshgrid(np.arange(n), np.arange(n), indexing="xy")
    phi = np.tanh((9 - np.sqrt((x - 19.5) ** 2 + (y - 19.5) ** 2)) / 1.5).ravel()
    rr, rb = (1 + phi) / 2, (1 - phi) / 2
    plain = oracle.make_cg_cfg("D2Q9", (n, n), 0.9, 0.01, 0.7)
    fr, fb = oracle.cg_init(plain, rr, rb)
    ref = oracle.cg_run(plain, fr, fb, 30)
    for amp in (0.0, 0.05):
        cfg = oracle.make_cg_cfg("D2Q9", (n, n), 0.9, 0.01, 0.7, nci_amp=amp, nci_eps=0.1, nci_h=2)
        out = oracle.cg_run(cfg, fr, fb, 30)
        assert np.array_equal(out[0], ref[0]) and np.array_equal(out[1], ref[1])


@pytest.mark.parametrize("lat", ["D2Q9", "D3Q19"])
def test_nci_momentum_change_equals_sum_of_forces(lat):
    """The repulsion is a body force: over one step the total momentum of
    the two colours changes by exactly the sum over flagged nodes of
    A rho_R grad phi / |grad phi| (flags and gradient pinned above; the
    perturbation, recolouring and streaming conserve momentum).  Unequal
    droplets, so that the forces do not cancel."""
    amp = 0.02
    if lat == "D2Q9":
        n, d = 32, 2
        phi = _two_spheres(n, 9.0, 3.0, d=2, R2=6.0)
        dims = (2 * n, n)
    else:
        n, d = 16, 3
        phi = _two_spheres(n, 5.0, 3.0, R2=4.0)
        dims = (2 * n, n, n)
    cfg = oracle.make_cg_cfg(lat, dims, 0.9, 0.01, 0.7, nci_amp=amp, nci_eps=0.1, nci_h=2)
    fr, fb = oracle.cg_init(cfg, (1 + phi) / 2, (1 - phi) / 2)
    fr, fb = oracle.cg_run(cfg, fr, fb, 20)
    R0, B0, u0 = oracle.cg_fields(cfg, fr, fb)
    ph = (R0 - B0) / (R0 + B0)
    fl = oracle.cg_nci_flags(cfg, ph)
    g = oracle.cg_gradient(cfg, ph)
    gn = np.sqrt((g ** 2).sum(0))
    F = np.where((fl > 0) & (gn > 0), amp * R0 / np.where(gn > 0, gn, 1.0), 0.0) * g
    assert fl.sum() > 0 and np.abs(F.sum(1)).max() > 1e-4
    R1, B1, u1 = oracle.cg_fields(cfg, *oracle.cg_run(cfg, fr, fb, 1))
    assert np.abs(cfg.rho0 * (u1 - u0).sum(1) - F.sum(1)).max() < 1e-13


def test_nci_repulsion_prevents_coalescence():
    """Two droplets driven towards each other coalesce without the
    near-contact force (the film between them fills with the dispersed
    phase) and stay apart with it (the film survives and the droplets are
    pushed apart): the sign and the effect of the section 2.2 force."""
    nx, ny, R, gap, U = 96, 48, 10.0, 6.0, 0.03
    x, y = np.meshgrid(np.arange(nx), np.arange(ny), indexing="xy")
    c1, c2, cy = nx / 2 - gap / 2 - R, nx / 2 + gap / 2 + R, (ny - 1) / 2
    phi = np.maximum(np.tanh((R - np.hypot(x - c1, y - cy)) / 1.5),
                     np.tanh((R - np.hypot(x - c2, y - cy)) / 1.5)).ravel()
    u = np.zeros((2, nx * ny))
    u[0] = np.where(x.ravel() < nx / 2, U, -U) * (phi > -0.5)
    X = np.tile(np.arange(nx), ny)
    left = X < nx / 2

    def run(amp):
        cfg = oracle.make_cg_cfg("D2Q9", (nx, ny), 1.0, 0.01, 0.7, nci_amp=amp, nci_eps=0.1, nci_h=2)
        fr, fb = oracle.cg_init(cfg, (1 + phi) / 2, (1 - phi) / 2, u)
        mid = []
        for _ in range(10):
            fr, fb = oracle.cg_run(cfg, fr, fb, 200)
            Rr, Bb, _ = oracle.cg_fields(cfg, fr, fb)
            mid.append(((Rr - Bb) / (Rr + Bb)).reshape(ny, nx)[ny // 2, nx // 2 - 1:nx // 2 + 1].max())
        sep = (Rr * X)[~left].sum() / Rr[~left].sum() - (Rr * X)[left].sum() / Rr[left].sum()
        return np.array(mid), sep

    mid0, sep0 = run(0.0)
    mid1, sep1 = run(0.01)
    assert mid0[-1] > 0.9                      # merged: the film is dispersed phase
    assert mid1.max() < -0.5                   # the film survives throughout
    assert sep1 > 2 * R + gap and sep1 > sep0 + 5
