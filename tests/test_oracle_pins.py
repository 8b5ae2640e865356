"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: textbook
lattice identities, the moments the He-Luo equilibrium must carry (Eq. equil),
the defining property of the order-2 Hermite projection (Eq. hermite and the
compact form of fhat^neq in section 3), the special cases where the
regularized step reduces to plain BGK (Eq. lbe), exact conservation, closed
form flows (Taylor-Green decay with nu = cs2 (1/omega - 1/2) from section 2;
the Poiseuille parabola) and an independent numpy brute force.
"""
import math

import numpy as np
import pytest

import oracle
import synth
from oracle.brute import BruteLB

LATTICES = ["D2Q9", "D3Q19", "D3Q27"]
CS2 = 1.0 / 3.0


def _dims(lat, n):
    return (n, n, 1) if lat == "D2Q9" else (n, n, n)


def _d(lat):
    return 2 if lat == "D2Q9" else 3


# ---------------------------------------------------------------- lattices
@pytest.mark.parametrize("lat,q", [("D2Q9", 9), ("D3Q19", 19), ("D3Q27", 27)])
def test_lattice_isotropy(lat, q):
    c, w, opp = oracle.lattice_tables(lat)
    d = _d(lat)
    c = c[:, :d].astype(float)
    assert len(w) == q
    assert abs(w.sum() - 1.0) < 1e-15
    assert np.abs(w @ c).max() < 1e-15
    assert np.abs(np.einsum("a,ai,aj->ij", w, c, c) - CS2 * np.eye(d)).max() < 1e-15
    # third moment vanishes, fourth is isotropic: cs2^2 (d_ij d_kl + d_ik d_jl + d_il d_jk)
    assert np.abs(np.einsum("a,ai,aj,ak->ijk", w, c, c, c)).max() < 1e-15
    I = np.eye(d)
    iso = CS2 ** 2 * (np.einsum("ij,kl->ijkl", I, I) + np.einsum("ik,jl->ijkl", I, I) + np.einsum("il,jk->ijkl", I, I))
    assert np.abs(np.einsum("a,ai,aj,ak,al->ijkl", w, c, c, c, c) - iso).max() < 1e-15
    # opposite table is an involution mapping c -> -c
    assert (opp[opp] == np.arange(q)).all()
    assert (c[opp] == -c).all()


@pytest.mark.parametrize("lat", LATTICES)
def test_lattice_order_and_tables_match_brute(lat):
    c, w, opp = oracle.lattice_tables(lat)
    cb, wb, oppb, _ = oracle.brute.lattice(lat)
    assert (c == cb).all() and np.allclose(w, wb, rtol=0, atol=1e-16) and (opp == oppb).all()
    # canonical order: rest first, |c|^2 non-decreasing, lexicographic inside a shell
    c2 = (c * c).sum(1)
    assert c2[0] == 0 and (np.diff(c2) >= 0).all()
    for s in np.unique(c2):
        rows = [tuple(r) for r in c[c2 == s]]
        assert rows == sorted(rows)


# ------------------------------------------------------------- equilibrium
@pytest.mark.parametrize("lat", LATTICES)
def test_equilibrium_moments(lat):
    """Eq. equil carries rho, rho0 u and rho cs2 I + rho0 u u (He & Luo)."""
    c, w, _ = oracle.lattice_tables(lat)
    d = _d(lat)
    g = synth.rng(1)
    for _ in range(5):
        rho0 = g.uniform(0.8, 1.2)
        cfg = oracle.make_cfg(lat, _dims(lat, 4), 0.8, rho0=rho0)
        rho = rho0 + g.uniform(-0.05, 0.05)
        u = g.uniform(-0.1, 0.1, size=d)
        feq = oracle.equilibrium(cfg, rho, u)
        cc = c[:, :d].astype(float)
        assert abs(feq.sum() - rho) < 1e-15
        assert np.abs(feq @ cc - rho0 * u).max() < 1e-15
        Pi = np.einsum("a,ai,aj->ij", feq, cc, cc)
        assert np.abs(Pi - (rho * CS2 * np.eye(d) + rho0 * np.outer(u, u))).max() < 1e-15


# ------------------------------------------------------ Hermite projection
@pytest.mark.parametrize("lat", LATTICES)
def test_regularizer_identities(lat):
    """fhat keeps the moments of order <= 2 (section 3: sum fhat c c = Pi^neq),
    is idempotent, and leaves span elements unchanged.  A wrong prefactor
    (e.g. 1/(2 cs2) instead of 1/(2 cs2^2)) breaks the second-moment check."""
    c, w, _ = oracle.lattice_tables(lat)
    d = _d(lat)
    cc = c[:, :d].astype(float)
    g = synth.uniform_noise(len(w), seed=7) * 1e-2
    gh = oracle.project_neq(lat, g)
    assert abs(gh.sum() - g.sum()) < 1e-16
    assert np.abs(gh @ cc - g @ cc).max() < 1e-16
    assert np.abs(np.einsum("a,ai,aj->ij", gh, cc, cc) - np.einsum("a,ai,aj->ij", g, cc, cc)).max() < 1e-16
    assert np.abs(oracle.project_neq(lat, gh) - gh).max() < 1e-17
    # an arbitrary set is not in the span (the projection really filters)
    assert np.abs(gh - g).max() > 1e-4
    # the residual is orthogonal to the span in <x, y> = sum x y / w
    brute = BruteLB(lat, _dims(lat, 2), 0.8)
    assert np.abs(brute.H.T @ (g - gh)).max() < 1e-16


@pytest.mark.parametrize("lat", LATTICES)
def test_pineq_matches_definition(lat):
    """Pi^neq returned by the collision equals sum (f - f^eq) c c (section 4)."""
    c, w, _ = oracle.lattice_tables(lat)
    d = _d(lat)
    cfg = oracle.make_cfg(lat, _dims(lat, 4), 0.7)
    f = w * (1.0 + 0.05 * synth.uniform_noise(len(w), seed=3))
    _, pineq = oracle.collide_node(cfg, f)
    cc = c[:, :d].astype(float)
    rho = f.sum()
    u = f @ cc
    feq = oracle.equilibrium(cfg, rho, u)
    P = np.einsum("a,ai,aj->ij", f - feq, cc, cc)
    if d == 2:
        ref = [P[0, 0], P[1, 1], P[0, 1]]
    else:
        ref = [P[0, 0], P[1, 1], P[2, 2], P[0, 1], P[0, 2], P[1, 2]]
    assert np.abs(pineq - ref).max() < 1e-16


# --------------------------------------- reductions to plain BGK (Eq. lbe)
@pytest.mark.parametrize("lat", LATTICES)
def test_tau_one_is_equilibrium_streaming(lat):
    """At omega = 1 Eq. LBexp gives f* = f^eq: one step equals pushing the
    equilibrium of every node one link along c_a (textbook BGK at tau = 1)."""
    dims = _dims(lat, 6)
    d = _d(lat)
    cfg = oracle.make_cfg(lat, dims, 1.0)
    rho, u, pineq = synth.smooth_random_state(dims, d, seed=11)
    f0 = oracle.init(cfg, rho, u, pineq) + 1e-3 * synth.uniform_noise((len(oracle.lattice_tables(lat)[1]), rho.size), seed=12)
    f1 = oracle.run(cfg, f0, 1)
    c, w, _ = oracle.lattice_tables(lat)
    r0, u0 = oracle.moments(cfg, f0)
    nx, ny, nz = dims
    for a in range(len(w)):
        feq_a = np.array([oracle.equilibrium(cfg, r0[i], u0[:, i])[a] for i in range(r0.size)])
        pushed = np.roll(feq_a.reshape(nz, ny, nx), shift=(c[a, 2], c[a, 1], c[a, 0]), axis=(0, 1, 2))
        assert np.abs(pushed.reshape(-1) - f1[a]).max() < 1e-15


@pytest.mark.parametrize("lat", LATTICES)
def test_hermite_span_state_is_plain_bgk(lat):
    """If f^neq already lies in the order-2 Hermite span the projection is the
    identity, so the regularized collision equals BGK f + omega (f^eq - f)."""
    c, w, _ = oracle.lattice_tables(lat)
    d = _d(lat)
    tau = 0.63
    cfg = oracle.make_cfg(lat, _dims(lat, 4), tau)
    g = synth.rng(5)
    rho, u = 1.0 + g.uniform(-0.02, 0.02), g.uniform(-0.05, 0.05, size=d)
    feq = oracle.equilibrium(cfg, rho, u)
    P = g.uniform(-1e-3, 1e-3, size=(d, d))
    P = P + P.T
    cc = c[:, :d].astype(float)
    fneq = w * (np.einsum("ai,aj,ij->a", cc, cc, P) - CS2 * np.trace(P)) / (2 * CS2 * CS2)
    f = feq + fneq
    fpc, _ = oracle.collide_node(cfg, f)
    bgk = f + (1.0 / tau) * (feq - f)
    assert np.abs(fpc - bgk).max() < 1e-15
    # and a state with higher-order content differs from BGK
    f2 = f + 1e-3 * w * synth.uniform_noise(len(w), seed=6)
    fpc2, _ = oracle.collide_node(cfg, f2)
    r2 = f2.sum()
    u2 = f2 @ cc
    bgk2 = f2 + (1.0 / tau) * (oracle.equilibrium(cfg, r2, u2) - f2)
    assert np.abs(fpc2 - bgk2).max() > 1e-6


# ---------------------------------------------------------- streaming pin
@pytest.mark.parametrize("lat", LATTICES)
def test_stream_is_pull_of_collided_set(lat):
    """One periodic step moves each collided population one link along c_a."""
    dims = _dims(lat, 5)
    d = _d(lat)
    cfg = oracle.make_cfg(lat, dims, 0.71)
    rho, u, pineq = synth.smooth_random_state(dims, d, seed=21)
    f0 = oracle.init(cfg, rho, u, pineq)
    f0 = f0 + 1e-3 * synth.uniform_noise(f0.shape, seed=22) * oracle.lattice_tables(lat)[1][:, None]
    f1 = oracle.run(cfg, f0, 1)
    c, w, _ = oracle.lattice_tables(lat)
    fpc = np.stack([oracle.collide_node(cfg, f0[:, i])[0] for i in range(f0.shape[1])], axis=1)
    nx, ny, nz = dims
    for a in range(len(w)):
        pushed = np.roll(fpc[a].reshape(nz, ny, nx), shift=(c[a, 2], c[a, 1], c[a, 0]), axis=(0, 1, 2))
        assert np.abs(pushed.reshape(-1) - f1[a]).max() < 1e-15


# ------------------------------------------------------------ conservation
@pytest.mark.parametrize("lat,n,steps", [("D2Q9", 24, 400), ("D3Q19", 10, 150), ("D3Q27", 8, 150)])
def test_conservation_periodic(lat, n, steps):
    dims = _dims(lat, n)
    d = _d(lat)
    cfg = oracle.make_cfg(lat, dims, 0.57)
    rho, u, pineq = synth.smooth_random_state(dims, d, seed=31)
    f = oracle.init(cfg, rho, u, pineq)
    c, w, _ = oracle.lattice_tables(lat)
    M0, J0 = f.sum(), (c[:, :d].T @ f).sum(axis=1)
    f = oracle.run(cfg, f, steps)
    M1, J1 = f.sum(), (c[:, :d].T @ f).sum(axis=1)
    N = rho.size
    assert abs(M1 - M0) / M0 < 1e-13
    assert np.abs(J1 - J0).max() <= 1e-13 * N


@pytest.mark.parametrize("lat", LATTICES)
def test_force_adds_exact_momentum(lat):
    """With a body force F every step adds exactly F per node (periodic box)."""
    dims = _dims(lat, 6)
    d = _d(lat)
    F = (2e-5, -1e-5, 3e-5)[:d] + (0.0,) * (3 - d)
    cfg = oracle.make_cfg(lat, dims, 0.9, force=F)
    rho, u, pineq = synth.smooth_random_state(dims, d, seed=41)
    f = oracle.init(cfg, rho, u, pineq)
    c, _, _ = oracle.lattice_tables(lat)
    J0 = (c[:, :d].T @ f).sum(axis=1)
    steps = 20
    f = oracle.run(cfg, f, steps)
    J1 = (c[:, :d].T @ f).sum(axis=1)
    N = rho.size
    assert np.abs((J1 - J0) - steps * N * np.array(F[:d])).max() < 1e-14 * N
    assert abs(f.sum() - rho.sum()) < 1e-12


@pytest.mark.parametrize("lat", LATTICES)
@pytest.mark.parametrize("faces", [[1] * 6, [0, 0, 1, 1, 0, 0], [1, 1, 0, 0, 1, 1]])
def test_rest_state_is_fixed_point(lat, faces):
    dims = _dims(lat, 5)
    d = _d(lat)
    if d == 2:
        faces = faces[:4] + [0, 0]
    cfg = oracle.make_cfg(lat, dims, 0.8, faces=faces)
    rho, u = synth.rest_state(dims, d)
    f0 = oracle.init(cfg, rho, u)
    f1 = oracle.run(cfg, f0, 50)
    assert np.abs(f1 - f0).max() < 1e-15


@pytest.mark.parametrize("lat", LATTICES)
def test_uniform_flow_is_fixed_point(lat):
    dims = _dims(lat, 5)
    d = _d(lat)
    cfg = oracle.make_cfg(lat, dims, 0.8)
    rho, u = synth.rest_state(dims, d)
    u[:] = np.array([0.03, -0.02, 0.01][:d])[:, None]
    f0 = oracle.init(cfg, rho, u)
    f1 = oracle.run(cfg, f0, 20)
    assert np.abs(f1 - f0).max() < 1e-15


@pytest.mark.parametrize("lat", LATTICES)
def test_moving_lid_momentum_injection(lat):
    """From rest, one step next to a lid moving at U along x adds x-momentum
    rho0 U cs2 per lid node (halfway bounce-back with the moving-wall term;
    sum over links of 2 t_a c_ax^2 rho0 U / cs2 = rho0 U cs2 by isotropy)."""
    n = 6
    dims = _dims(lat, n)
    d = _d(lat)
    U = 0.05
    rho0 = 1.1
    faces = [0, 0, 1, 2, 0, 0]  # periodic x (and z), stationary -y, lid +y
    wall_u = [[0, 0, 0]] * 3 + [[U, 0, 0]] + [[0, 0, 0]] * 2
    cfg = oracle.make_cfg(lat, dims, 0.7, rho0=rho0, faces=faces, wall_u=wall_u)
    rho, u = synth.rest_state(dims, d, rho0=rho0)
    f0 = oracle.init(cfg, rho, u)
    f1 = oracle.run(cfg, f0, 1)
    c, _, _ = oracle.lattice_tables(lat)
    dJ = (c[:, :d].T @ (f1 - f0)).sum(axis=1)
    lid_nodes = n if d == 2 else n * n
    assert abs(dJ[0] - lid_nodes * rho0 * U * CS2) < 1e-15
    assert np.abs(dJ[1:]).max() < 1e-15
    assert abs(f1.sum() - f0.sum()) < 1e-14 * f0.sum()


# ------------------------------------------------------ brute-force parity
CASES = [
    ("periodic", [0] * 6, None, (0, 0, 0)),
    ("walls", [1] * 6, None, (0, 0, 0)),
    ("lid", [1, 1, 1, 2, 1, 1], [[0, 0, 0]] * 3 + [[0.05, 0, 0]] + [[0, 0, 0]] * 2, (0, 0, 0)),
    ("duct_forced", [0, 0, 1, 1, 1, 1], None, (1e-4, 0, 0)),
    ("lid_periodic_z", [1, 1, 1, 2, 0, 0], [[0, 0, 0]] * 3 + [[0.04, 0, 0.01]] + [[0, 0, 0]] * 2, (0, 2e-5, 0)),
]


@pytest.mark.parametrize("lat", LATTICES)
@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_c_oracle_matches_brute_force(lat, case):
    name, faces, wall_u, force = case
    d = _d(lat)
    dims = (7, 6, 1) if d == 2 else (5, 4, 3)
    if d == 2:
        faces = faces[:4] + [0, 0]
    cfg = oracle.make_cfg(lat, dims, 0.62, rho0=1.0, force=force, faces=faces, wall_u=wall_u)
    rho, u, pineq = synth.smooth_random_state(dims, d, seed=51)
    f0 = oracle.init(cfg, rho, u, pineq)
    w = oracle.lattice_tables(lat)[1]
    f0 = f0 + 2e-3 * w[:, None] * synth.uniform_noise(f0.shape, seed=52)
    brute = BruteLB(lat, dims, 0.62, rho0=1.0, force=force, faces=faces, wall_u=wall_u)
    steps = 3
    fb = brute.run(f0, steps)
    fo = oracle.run(cfg, f0, steps)
    assert np.abs(fb - fo).max() < 1e-15
    rb, ub = brute.moments(fb)
    ro, uo = oracle.moments(cfg, fo)
    assert np.abs(rb - ro).max() < 1e-14 and np.abs(ub - uo).max() < 1e-15


@pytest.mark.slow
@pytest.mark.parametrize("lat", ["D3Q19", "D3Q27"])
def test_c_oracle_matches_brute_force_8cubed(lat):
    """The 8^3 one-step and ten-step brute-force comparison."""
    dims = (8, 8, 8)
    faces = [1, 1, 1, 2, 0, 0]
    wall_u = [[0, 0, 0]] * 3 + [[0.05, 0, 0]] + [[0, 0, 0]] * 2
    cfg = oracle.make_cfg(lat, dims, 0.55, faces=faces, wall_u=wall_u)
    rho, u, pineq = synth.smooth_random_state(dims, 3, seed=61)
    f0 = oracle.init(cfg, rho, u, pineq)
    brute = BruteLB(lat, dims, 0.55, faces=faces, wall_u=wall_u)
    f1b = brute.step(f0)
    assert np.abs(f1b - oracle.run(cfg, f0, 1)).max() < 1e-15
    f10b = brute.run(f1b, 9)
    assert np.abs(f10b - oracle.run(cfg, f0, 10)).max() < 1e-14


# ------------------------------------------------------------ closed forms
def _tg_decay_rate(lat, n, tau, u0, t0, t1, stride):
    """Fitted viscosity from the decay of the vortex amplitude: the 2D vortex
    has |k|^2 = 2 k^2, the 3D one |k|^2 = 3 k^2 (amplitude ~ exp(-nu |k|^2 t))."""
    if lat == "D2Q9":
        dims = (n, n, 1)
        rho, u, pineq = synth.taylor_green_2d(n, u0=u0, tau=tau)
        mode = synth.taylor_green_2d_mode(n)
        kk = 2
    else:
        dims = (n, n, n)
        rho, u, pineq = synth.taylor_green_3d(n, u0=u0, tau=tau)
        mode = u / u0
        kk = 3
    cfg = oracle.make_cfg(lat, dims, tau)
    f = oracle.init(cfg, rho, u, pineq)
    f = oracle.run(cfg, f, t0)
    ts, amps = [], []
    t = t0
    while t <= t1:
        _, uu = oracle.moments(cfg, f)
        amps.append((uu * mode).sum() / (mode * mode).sum())
        ts.append(t)
        f = oracle.run(cfg, f, stride)
        t += stride
    slope = np.polyfit(np.array(ts, float), np.log(np.array(amps)), 1)[0]
    k = 2 * math.pi / n
    return -slope / (kk * k * k)  # fitted nu


@pytest.mark.slow
def test_taylor_green_2d_decay_rate():
    """Velocity amplitude of the 256^2 vortex (u0 = 0.01, tau = 0.8) decays as
    exp(-2 nu k^2 t) with nu = cs2 (1/omega - 1/2) (section 2); fit 100..1000."""
    tau = 0.8
    nu_fit = _tg_decay_rate("D2Q9", 256, tau, 0.01, 100, 1000, 100)
    nu = CS2 * (tau - 0.5)
    assert abs(nu_fit / nu - 1) < 2e-4  # measured 6e-5


@pytest.mark.parametrize("lat", ["D3Q19", "D3Q27"])
def test_taylor_green_3d_decay_rate(lat):
    tau = 0.8
    nu_fit = _tg_decay_rate(lat, 24, tau, 0.01, 20, 200, 20)
    nu = CS2 * (tau - 0.5)
    # 24 nodes per wavelength: the lattice error is O(k^2), a few 1e-3
    assert abs(nu_fit / nu - 1) < 1e-2


def _poiseuille_error(lat, H, tau, F):
    d = _d(lat)
    dims = (1, H, 1)
    faces = [0, 0, 1, 1, 0, 0]
    nu = CS2 * (tau - 0.5)
    cfg = oracle.make_cfg(lat, dims, tau, force=(F, 0, 0), faces=faces)
    rho, u = synth.channel_state(dims, F, 1.0, nu, d)
    f = oracle.init(cfg, rho, u)
    steps = int(6 * H * H / (math.pi ** 2 * nu))
    f = oracle.run(cfg, f, steps)
    f2 = oracle.run(cfg, f, 200)
    _, u1 = oracle.moments(cfg, f)
    _, u2 = oracle.moments(cfg, f2)
    assert np.abs(u2 - u1).max() < 1e-6 * np.abs(u2).max()  # steady
    ana = synth.poiseuille_profile(H, F, 1.0, nu)
    return np.linalg.norm(u2[0] - ana) / np.linalg.norm(ana), np.abs(u2[1:]).max()


@pytest.mark.parametrize("lat", LATTICES)
def test_poiseuille_parabola_second_order(lat):
    tau, F = 0.6, 1e-6
    e16, v16 = _poiseuille_error(lat, 16, tau, F)
    e32, v32 = _poiseuille_error(lat, 32, tau, F)
    assert v16 < 1e-12 and v32 < 1e-12
    assert e32 < 5e-3
    assert 3.5 < e16 / e32 < 4.5


# ---------------------------------------------------------------- reduced-precision storage
def test_storage_rounding_fp16_is_ieee_binary16():
    """Round-to-nearest-even to binary16, pinned against hand-made ties and
    numpy's own float64 -> float16 conversion (normal and subnormal range)."""
    from oracle.storage import quantum, round_to_format
    ties = np.array([1 + 2.0 ** -11, 1 + 3 * 2.0 ** -11, -(1 + 2.0 ** -11), 2.0 ** -24 * 0.5, 2.0 ** -24 * 1.5,
                     2.0 ** -14 + 2.0 ** -25, 0.0])
    want = np.array([1.0, 1 + 2.0 ** -9, -1.0, 0.0, 2.0 ** -23, 2.0 ** -14, 0.0])
    assert np.array_equal(round_to_format(ties, "f16s"), want)
    g = synth.rng(5)
    for scale in (1e-1, 3e-3, 1e-5, 1e-7):
        x = g.uniform(-scale, scale, size=20000)
        assert np.array_equal(round_to_format(x, "f16s"), x.astype(np.float16).astype(np.float64))
    assert quantum(np.array([1.0, 1.5, 2.0 ** -20]), "f16s").tolist() == [2.0 ** -10, 2.0 ** -10, 2.0 ** -24]


def test_storage_rounding_bf16_is_round_to_nearest_even():
    """bfloat16 keeps 8 significant bits with the FP32 exponent range; pinned
    against hand-made ties and torch's float32 -> bfloat16 conversion on
    values that FP32 represents exactly."""
    torch = pytest.importorskip("torch")
    from oracle.storage import round_to_format
    ties = np.array([1 + 2.0 ** -8, 1 + 3 * 2.0 ** -8, -(1 + 2.0 ** -8), 2.0 ** -20 * (1 + 2.0 ** -9)])
    want = np.array([1.0, 1 + 2.0 ** -6, -1.0, 2.0 ** -20])
    assert np.array_equal(round_to_format(ties, "bf16s"), want)
    g = synth.rng(6)
    for scale in (1e-1, 3e-3, 1e-5):
        x = g.uniform(-scale, scale, size=20000).astype(np.float32)
        ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
        assert np.array_equal(round_to_format(x.astype(np.float64), "bf16s"), ref)


def test_stored_run_shifts_before_rounding():
    """The reduced modes round f_a - t_a rho0, so a rest state (f = t_a rho0)
    is stored exactly and stays at rest (up to FP64 rounding) in every format."""
    from oracle.storage import round_populations
    cfg = oracle.make_cfg("D3Q19", (4, 3, 5), 0.7, rho0=1.0)
    rho, u = synth.rest_state((4, 3, 5), 3)
    f0 = oracle.init(cfg, rho, u)
    w = oracle.lattice_tables("D3Q19")[1]
    for st in ("f16s", "bf16s", "f32"):
        assert np.array_equal(round_populations(f0, w, st), f0)
        assert np.abs(oracle.run_stored(cfg, f0, 3, st) - f0).max() < 1e-15
    # without the shift binary16 could not hold t_a = 1/36 exactly
    from oracle.storage import round_to_format
    assert round_to_format(np.array([1.0 / 36.0]), "f16s")[0] != 1.0 / 36.0
