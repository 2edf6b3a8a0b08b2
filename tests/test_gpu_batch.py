"""Batched engine (many uneven systems per launch, one CUDA graph per step) against
the per-system C-ABI path and the CPU oracle.

The batched step computes the same predictor-corrector Magnus step (Sec. VI.B) as
tdks_magnus_step; only the grouping of partial sums differs (element and row
blocks), so FP64 orbitals agree to rounding unless a Krylov stopping index sits on
a tie, which moves results by at most the Lanczos tolerance: the bound is 1e-10
relative, the orbital tolerance of the FP64 path.
"""
import numpy as np
import pytest

import synth
from oracle.mesh import Mesh
from oracle.propagate import Propagator, kick

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1810_13130_gb300.build import build
    build()


def _rel(a, b):
    return float(np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(b).max(), 1e-300))


def _initial(cfgs):
    out = []
    for k, c in enumerate(cfgs):
        ni = tuple((len(a) - 1) * c.p - 1 for a in (c.X, c.Y, c.Z))
        out.append(synth.smooth_orbitals(ni, c.n_orb, seed=100 + k))
    return out


def _batch(cfgs, psi0, prec=0, tol=1e-10, k_max=64):
    from paper_1810_13130_gb300 import tdks
    b = tdks.Batch(cfgs, [c.dt for c in cfgs], prec=prec, tol=tol, k_max=k_max)
    for k, p in enumerate(psi0):
        b.set_orbitals(k, torch.from_numpy(p).cuda())
    b.kick([c.kick for c in cfgs], [c.kick_dir for c in cfgs])
    d0 = b.init()
    return b, d0


def _per_system(cfg, psi0, n_steps, prec=0):
    from paper_1810_13130_gb300 import tdks
    ctx = tdks.Context.from_config(cfg)
    g = torch.from_numpy(psi0).cuda()
    ctx.kick(g, cfg.kick, cfg.kick_dir)
    d0 = ctx.init_propagation(g)
    dips = [ctx.magnus_step(g, cfg.dt, tol=1e-10, k_max=64, prec=prec)["dipole"] for _ in range(n_steps)]
    return g.cpu().numpy(), d0, np.array(dips)


def test_batch_fp64_matches_per_system_path():
    cfgs = synth.small_batch()
    psi0 = _initial(cfgs)
    b, d0 = _batch(cfgs, psi0)
    n = 3
    dips = b.steps(n)
    assert dips.shape == (n, len(cfgs), 3)
    for k, c in enumerate(cfgs):
        ref, r0, rd = _per_system(c, psi0[k], n)
        np.testing.assert_allclose(d0[k], r0, rtol=1e-12, atol=1e-14)
        assert _rel(b.get_orbitals(k).cpu().numpy(), ref) < 1e-10
        ind = max(np.abs(rd - r0).max(), 1e-300)
        assert np.abs(dips[:, k] - rd).max() <= 1e-9 * ind + 1e-14


def test_batch_matches_oracle():
    cfgs = synth.small_batch()[:4]
    psi0 = _initial(cfgs)
    b, _ = _batch(cfgs, psi0)
    n = 2
    dips = b.steps(n)
    for k, c in enumerate(cfgs):
        m = Mesh.from_config(c)
        prop = Propagator.from_config(c, m)
        ref = kick(m, psi0[k], c.kick, c.kick_dir)
        prop.init(ref)
        for s in range(n):
            ref, dref, _ = prop.magnus_step(ref, c.dt)
            np.testing.assert_allclose(dips[s, k], dref, rtol=1e-9, atol=1e-12)
        assert _rel(b.get_orbitals(k).cpu().numpy(), ref) < 1e-10


@pytest.mark.parametrize("prec,bound", [(2, 1e-10), (1, 1e-5)])
def test_batch_mixed_precision_vs_fp64(prec, bound):
    cfgs = synth.small_batch()
    psi0 = _initial(cfgs)
    b, _ = _batch(cfgs, psi0, prec=prec)
    b.steps(2)
    for k, c in enumerate(cfgs):
        ref, _, _ = _per_system(c, psi0[k], 2)
        assert _rel(b.get_orbitals(k).cpu().numpy(), ref) < bound


def test_batch_tuned_tiles_give_the_same_step():
    cfgs = synth.small_batch()
    psi0 = _initial(cfgs)
    a, _ = _batch(cfgs, psi0)
    b, _ = _batch(cfgs, psi0)
    tiles = b.tune(reps=2)
    assert {(t["p"], t["n_orb"]) for t in tiles} == {(c.p, c.n_orb) for c in cfgs}
    for t in tiles:
        assert 1 <= t["elems_per_cta"] <= 256 // (t["p"] + 1) ** 2
        assert 1 <= t["orbs_per_item"] <= t["n_orb"]
    da, db = a.steps(3), b.steps(3)
    np.testing.assert_allclose(db, da, rtol=1e-11, atol=1e-15)
    for k in range(len(cfgs)):
        assert _rel(b.get_orbitals(k).cpu().numpy(), a.get_orbitals(k).cpu().numpy()) < 1e-11


def test_batch_replays_are_independent_of_the_step_chunking():
    cfgs = synth.small_batch()[:3]
    psi0 = _initial(cfgs)
    a, _ = _batch(cfgs, psi0)
    b, _ = _batch(cfgs, psi0)
    da = a.steps(4)
    db = np.concatenate([b.steps(1), b.steps(3)])
    np.testing.assert_array_equal(da, db)
    st = a.stats()
    assert st["dof_applies"] > 0 and 1 <= st["k_max_seen"] <= 64


def test_batch_workload_subset_full_size():
    """Eight systems of the 64-system batch workload (sizes up to 12^3 elements,
    p up to 8): two batched steps against the per-system path."""
    cfgs, dts, dirs = synth.config5()
    pick = [int(i) for i in np.argsort([-(len(c.X) - 1) ** 3 * c.p ** 3 * c.n_orb for c in cfgs])[:2]]
    pick += [i for i in range(len(cfgs)) if i not in pick][:6]
    sub = [cfgs[i] for i in pick]
    psi0 = _initial(sub)
    b, _ = _batch(sub, psi0)
    b.tune(reps=1)
    dips = b.steps(2)
    for k, c in enumerate(sub):
        _, r0, rd = _per_system(c, psi0[k], 2)
        ind = max(np.abs(rd - r0).max(), 1e-300)
        assert np.abs(dips[:, k] - rd).max() <= 1e-9 * ind + 1e-13


def test_batch_rejects_bad_arguments():
    from paper_1810_13130_gb300 import tdks
    cfgs = synth.small_batch()[:2]
    with pytest.raises(tdks.TDKSError):
        tdks.Batch(cfgs, [0.05, -1.0])
    with pytest.raises(tdks.TDKSError):
        tdks.Batch(cfgs, [0.05, 0.1], prec=tdks.BF16)   # accuracy-study mode: single systems only
    b = tdks.Batch(cfgs, [0.05, 0.1])
    with pytest.raises(tdks.TDKSError):
        b.steps(1)                                   # no init yet
    with pytest.raises(tdks.TDKSError):
        b.set_orbitals(0, torch.zeros(1, 3, dtype=torch.complex128, device="cuda"))


def test_batch_krylov_caps_follow_the_substeps():
    """tdks_batch_tune_kmax raises the Krylov cap of exactly the systems whose
    exponential restarted at the cap (the per-system path at the same cap takes
    sub-steps there), within the memory budget; the steps after it equal the
    per-system path run with the same per-system caps."""
    from paper_1810_13130_gb300 import tdks
    cfgs = synth.small_batch()
    psi0 = _initial(cfgs)
    K0, K1 = 6, 16
    b, d0 = _batch(cfgs, psi0, k_max=K0)
    with pytest.raises(tdks.TDKSError):
        b.tune_kmax(K1)                              # no step yet: nothing to go by
    d1 = b.steps(1)
    # which systems restart at K0: the per-system path's own sub-step count
    ctxs, gs, subs = [], [], []
    for k, c in enumerate(cfgs):
        ctx = tdks.Context.from_config(c)
        g = torch.from_numpy(psi0[k]).cuda()
        ctx.kick(g, c.kick, c.kick_dir)
        ctx.init_propagation(g)
        st = ctx.magnus_step(g, c.dt, tol=1e-10, k_max=K0)
        subs.append(st["substeps"] > 0)
        ctxs.append(ctx)
        gs.append(g)
    assert any(subs) and not all(subs)
    assert b.tune_kmax(K1, mem_budget=0) == [K0] * len(cfgs)
    need = [c.n_orb * ((len(c.X) - 1) * c.p - 1) * ((len(c.Y) - 1) * c.p - 1) * ((len(c.Z) - 1) * c.p - 1)
            * (K1 - K0) * 16 for c in cfgs]
    total = sum(n for n, s in zip(need, subs) if s)
    if sum(subs) > 1:
        short = b.tune_kmax(K1, mem_budget=total - 1)  # one of them no longer fits
        assert 0 < sum(k == K1 for k in short) < sum(subs)
    caps = b.tune_kmax(K1, mem_budget=total)
    assert caps == [K1 if s else K0 for s in subs]
    dips = b.steps(2)
    for k, c in enumerate(cfgs):
        ref = [ctxs[k].magnus_step(gs[k], c.dt, tol=1e-10, k_max=caps[k]) for _ in range(2)]
        assert _rel(b.get_orbitals(k).cpu().numpy(), gs[k].cpu().numpy()) < 1e-10
        rd = np.array([r["dipole"] for r in ref])
        ind = max(np.abs(rd - d0[k]).max(), 1e-300)
        assert np.abs(dips[:, k] - rd).max() <= 1e-9 * ind + 1e-14
        if caps[k] == K1:
            assert all(r["substeps"] == 0 for r in ref) or max(r["k_full_max"] for r in ref) > K0
        ctxs[k].close()
    with pytest.raises(tdks.TDKSError):
        b.tune_kmax(200)


KB_ATOMS = {0: np.array([[0.3, -0.2, 0.1], [-2.1, 1.4, 0.9]]), 2: np.array([[0.3, -0.2, 0.1]])}


@pytest.mark.parametrize("prec_name,bound", [("fp64", 1e-10), ("df64", 1e-10), ("mixed", 1e-6)])
def test_batch_nonlocal_term_matches_oracle(prec_name, bound):
    """tdks_batch_set_kb on two systems of a batch (Eq. 6 in Galerkin and Loewdin form;
    one of them with three orbitals, so that each orbital projects its own Krylov
    vector): the batched steps equal the oracle's Magnus steps with the same
    projectors, and the systems without projectors stay as they were."""
    from paper_1810_13130_gb300 import tdks
    from oracle.kb import KleinmanBylander
    prec = {"fp64": tdks.FP64, "df64": tdks.DF64, "mixed": tdks.MIXED}[prec_name]
    cfgs = synth.small_batch()[:4]
    psi0 = _initial(cfgs)
    kp = synth.KBParams()
    b, _ = _batch(cfgs, psi0, prec=prec)
    for k, R in KB_ATOMS.items():
        b.set_kb(k, R, kp.a, kp.b, kp.c, kp.lmax)
    plain, _ = _batch(cfgs, psi0, prec=prec)
    n = 2
    dips, dplain = b.steps(n), plain.steps(n)
    for k, c in enumerate(cfgs):
        m = Mesh.from_config(c)
        nl = KleinmanBylander(m, KB_ATOMS[k], kp.a, kp.b, kp.c, lmax=kp.lmax) if k in KB_ATOMS else None
        prop = Propagator.from_config(c, m, nl=nl)
        ref = kick(m, psi0[k], c.kick, c.kick_dir)
        prop.init(ref)
        for s in range(n):
            ref, dref, _ = prop.magnus_step(ref, c.dt)
            np.testing.assert_allclose(dips[s, k], dref, rtol=1e-8 if bound > 1e-10 else 1e-9, atol=1e-12)
        got = b.get_orbitals(k).cpu().numpy()
        assert _rel(got, ref) < bound
        if k in KB_ATOMS:
            assert _rel(got, plain.get_orbitals(k).cpu().numpy()) > 1e-4   # the term acts
        else:
            np.testing.assert_array_equal(dips[:, k], dplain[:, k])


def test_batch_nonlocal_term_can_be_removed():
    cfgs = synth.small_batch()[:3]
    psi0 = _initial(cfgs)
    kp = synth.KBParams()
    a, _ = _batch(cfgs, psi0)
    b, _ = _batch(cfgs, psi0)
    b.set_kb(0, KB_ATOMS[0], kp.a, kp.b, kp.c, kp.lmax)
    b.set_kb(0, np.zeros((0, 3)))
    np.testing.assert_array_equal(b.steps(2), a.steps(2))


def test_batch_timing_and_profile_pass_are_diagnostics_only():
    """tdks_batch_set_timing / phase_ms / profile_pass: the timed graph gives the same
    steps bit for bit, the phase times and loop passes are reported, and the profile
    pass (the half-step exponential once more, kernel group by kernel group) leaves
    the orbitals as they were."""
    from paper_1810_13130_gb300 import tdks
    cfgs = synth.small_batch()[:3]
    psi0 = _initial(cfgs)
    a, _ = _batch(cfgs, psi0)
    b, _ = _batch(cfgs, psi0)
    with pytest.raises(tdks.TDKSError):
        b.profile_pass()                             # no step yet
    b.set_timing(True)
    with pytest.raises(tdks.TDKSError):
        b.phase_ms()
    np.testing.assert_array_equal(b.steps(2), a.steps(2))
    ph = b.phase_ms()
    assert all(ph[k] >= 0.0 for k in ("predictor", "half_exp", "corrector_fields", "full_exp",
                                       "history_dipole"))
    assert ph["half_exp"] > 0.0 and ph["full_exp"] > 0.0
    assert all(1 <= n <= 16 * 64 for n in ph["passes"])
    before = [b.get_orbitals(k).cpu().numpy() for k in range(len(cfgs))]
    pp = b.profile_pass()
    assert pp["apply"] > 0.0 and all(v >= 0.0 for v in pp.values())
    for k in range(len(cfgs)):
        np.testing.assert_array_equal(b.get_orbitals(k).cpu().numpy(), before[k])
    b.set_timing(False)
    np.testing.assert_array_equal(b.steps(1), a.steps(1))
