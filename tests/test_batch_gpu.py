"""Batched stepping (lb_batch_*) of many uneven domains.

A batch runs one persistent launch per brick-shape class and time step over a
static work list of all domains' bricks, replayed from a CUDA graph two steps
at a time.  Every domain must come out bit for bit equal to stepping it alone
(same per-node arithmetic, bricks and shells), for odd and even step counts,
with members that were also stepped alone in between, and with several
classes (lattices, storages, forcing) in one batch.  Every member is also
held directly to the CPU oracle: FP64 and FP32 members by the relative L2
error of rho and u (1e-12 / 1e-5), FP16 / BF16 members step by step within
one unit of the storage format of the rounded oracle step.
"""
import numpy as np
import pytest

import oracle
import synth
from lbcase import faces_for, oracle_cfg, random_state, rel_l2
from oracle.storage import quantum, round_populations

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lb():
    import torch
    assert torch.cuda.is_available()
    from paper_2304_06437_gb300 import build
    build.build()
    import paper_2304_06437_gb300 as P
    return P


def _specs(seed):
    """Uneven domains of two lattices, random sizes, tau, boundaries, storage."""
    g = synth.rng(seed)
    out = []
    for i in range(7):
        dims = tuple(int(v) for v in g.integers(5, 48, size=3))
        out.append(dict(lat="D3Q19", dims=dims, tau=float(g.uniform(0.55, 1.2)),
                        fname=["periodic", "lid", "walls", "duct"][i % 4], storage="f32"))
    for i in range(6):
        dims = (int(g.integers(8, 300)), int(g.integers(4, 120)), 1)
        out.append(dict(lat="D2Q9", dims=dims, tau=float(g.uniform(0.55, 1.2)),
                        fname=["periodic", "lid"][i % 2], storage="f32"))
    out.append(dict(lat="D3Q27", dims=(21, 13, 17), tau=0.7, fname="lid_periodic_z", storage="f32"))
    out.append(dict(lat="D3Q19", dims=(30, 11, 9), tau=0.6, fname="duct", storage="f16s"))
    out.append(dict(lat="D2Q9", dims=(77, 31, 1), tau=0.9, fname="lid", storage="bf16s"))
    out.append(dict(lat="D3Q19", dims=(19, 23, 10), tau=0.8, fname="lid", storage="f64"))
    return out


def _make(lb, spec, seed):
    faces, wall_u = faces_for(spec["lat"], spec["fname"])
    force = (2e-5, 1e-5, 0.0) if spec["fname"] == "duct" else (0, 0, 0)
    s = lb.Solver(spec["lat"], spec["dims"], spec["tau"], faces=faces, wall_u=wall_u, storage=spec["storage"],
                  force=force)
    s.set_populations(np.ascontiguousarray(random_state(spec["lat"], spec["dims"], seed)))
    return s


@pytest.mark.parametrize("steps", [1, 2, 7])
def test_batch_equals_solo_bitwise(lb, steps):
    specs = _specs(99)
    solo = []
    for i, sp in enumerate(specs):
        s = _make(lb, sp, 500 + i)
        s.step(steps)
        solo.append(s.get_populations())
        s.close()
    members = [_make(lb, sp, 500 + i) for i, sp in enumerate(specs)]
    with lb.Batch(members) as b:
        info = b.info()
        assert info["n_domains"] == len(specs)
        assert info["n_classes"] >= 5  # D3Q19, D3Q19 forced, D2Q9, D3Q27, f16s, bf16s ...
        b.step(steps)
        b.sync()
        for s, ref in zip(members, solo):
            assert np.array_equal(s.get_populations(), ref)
        assert info["launches_per_step"] == info["n_classes"]
    for s in members:
        s.close()


def test_batch_with_members_stepped_alone(lb):
    """Shell parities may differ between members: every other member takes a
    solo step between two batch calls; all must equal their solo runs."""
    specs = _specs(7)[:8]
    solo = []
    for i, sp in enumerate(specs):
        s = _make(lb, sp, 900 + i)
        s.step(3 + (1 if i % 2 == 0 else 0) + 4)
        solo.append(s.get_populations())
        s.close()
    members = [_make(lb, sp, 900 + i) for i, sp in enumerate(specs)]
    with lb.Batch(members) as b:
        b.step(3)
        for i, s in enumerate(members):
            if i % 2 == 0:
                s.step(1)  # alone, on the member's stream (which waits for the batch)
        b.step(4)
        b.sync()
        for s, ref in zip(members, solo):
            assert np.array_equal(s.get_populations(), ref)
    for s in members:
        s.close()


def test_batch_rejects_unsupported(lb):
    s2p = lb.Solver("D3Q19", (9, 9, 9), 0.7, storage="f32", scheme="two_pass")
    s32 = lb.Solver("D3Q19", (9, 9, 9), 0.7, storage="f32")
    for bad in ([s2p], [s32, s32], [s32, s2p]):
        with pytest.raises(lb.LBError):
            lb.Batch(bad)
    for s in (s2p, s32):
        s.close()


def test_batch_members_match_oracle(lb):
    """The batched kernel has its own argument table, work list and per-domain
    parity: each member is compared with the oracle run of its own input."""
    specs = _specs(99)
    f0s, cfgs, members = [], [], []
    for i, sp in enumerate(specs):
        faces, wall_u = faces_for(sp["lat"], sp["fname"])
        force = (2e-5, 1e-5, 0.0) if sp["fname"] == "duct" else (0, 0, 0)
        w = oracle.lattice_tables(sp["lat"])[1]
        # the stored initial state (set_populations rounds to the storage)
        f0s.append(round_populations(random_state(sp["lat"], sp["dims"], 500 + i), w, sp["storage"]))
        cfgs.append(oracle_cfg(sp["lat"], sp["dims"], sp["tau"], faces, wall_u, force=force))
        members.append(_make(lb, sp, 500 + i))
    prev = [f.copy() for f in f0s]
    with lb.Batch(members) as b:
        for step in range(3):
            b.step(1)
            b.sync()
            for sp, s, cfg, i in zip(specs, members, cfgs, range(len(specs))):
                if sp["storage"] not in ("f16s", "bf16s"):
                    continue
                w = oracle.lattice_tables(sp["lat"])[1]
                got = s.get_populations()
                ref = oracle.run_stored(cfg, prev[i], 1, sp["storage"])
                dg, dr = got - w[:, None], ref - w[:, None]
                ulp = np.maximum(quantum(dg, sp["storage"]), quantum(dr, sp["storage"]))
                assert (np.abs(dg - dr) <= ulp * (1 + 1e-12) + 1e-7).all(), (i, step)
                prev[i] = got
        b.step(4)
        b.sync()
        for sp, s, cfg, f0 in zip(specs, members, cfgs, f0s):
            if sp["storage"] not in ("f64", "f32"):
                continue
            r_ref, u_ref = oracle.moments(cfg, oracle.run(cfg, f0, 7))
            r, u = s.moments()
            tol = 1e-12 if sp["storage"] == "f64" else 1e-5
            assert rel_l2(r, r_ref) < tol and rel_l2(u, u_ref) < tol, (sp, rel_l2(r, r_ref), rel_l2(u, u_ref))
    for s in members:
        s.close()


def test_batched_reduction_equals_member_reductions(lb):
    """lb_batch_reduce: the same FP64 sums, residual history included, as
    lb_reduce on each member alone (bit for bit), over two rounds."""
    specs = _specs(13)
    a = [_make(lb, sp, 700 + i) for i, sp in enumerate(specs)]
    b = [_make(lb, sp, 700 + i) for i, sp in enumerate(specs)]
    with lb.Batch(a) as ba, lb.Batch(b) as bb:
        for rnd in range(2):
            ba.step(5)
            bb.step(5)
            got = ba.reduce(residual=True)
            bb.sync()
            want = [s.reduce(residual=True) for s in b]
            for g, w in zip(got, want):
                assert g["mass"] == w["mass"] and g["momentum"] == w["momentum"]
                assert g["residual"] == w["residual"] and not g["diverged"]
                if rnd == 0:
                    assert g["residual"] == 1.0
                else:
                    assert g["residual"] > 0.0 and g["residual"] != 1.0
        # without the residual: the history is left alone
        plain = ba.reduce()
        assert all("residual" not in r for r in plain)
    for s in a + b:
        s.close()


def test_batched_reduction_flags_only_the_diverged_member(lb):
    specs = _specs(5)[:4]
    members = [_make(lb, sp, 800 + i) for i, sp in enumerate(specs)]
    bad = members[2].get_populations()
    bad[3, 7] = np.nan
    members[2].set_populations(bad)
    with lb.Batch(members) as b:
        out = b.reduce()
        assert [r["diverged"] for r in out] == [False, False, True, False]
        want = [s.reduce() for i, s in enumerate(members) if i != 2]
        got = [r for i, r in enumerate(out) if i != 2]
        assert all(g["mass"] == w["mass"] for g, w in zip(got, want))
    for s in members:
        s.close()
