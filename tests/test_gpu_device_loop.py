"""The device-driven Lanczos loop (tdks_set_device_loop) against the host-driven one.

Both run the same kernels in the same order (Eqs. 36-38): the iterations of a
sub-step as conditional nodes of one CUDA graph launch, or launched one by one by
the host after it has read the Lanczos state.  The results must therefore be
identical bit for bit, for every contraction arithmetic, with sub-steps, with CGS2
re-orthogonalization and with the nonlocal term; and the device loop must read the
state once per sub-step instead of once per iteration.
"""
import numpy as np
import pytest

import synth
from oracle.mesh import Mesh
from oracle.propagate import kick

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1810_13130_gb300.build import build
    build()


NORMS = np.array([1.0, 1e-3, 1.0, 1e-6, 0.3, 1.0])


def _setup(tile=4):
    from paper_1810_13130_gb300 import tdks
    cfg = synth.small_config(3, 2, 3, p=5, n_orb=6, graded=True, seed=41)
    m = Mesh.from_config(cfg)
    ctx = tdks.Context.from_config(cfg)
    ctx.set_cg(1e-13)
    ctx.set_apply_tile(tile)
    v = synth.random_potential(m.n_elem * m.nq ** 3, seed=42).reshape(m.n_elem, -1)
    psi = synth.random_psi(6, m.N_int, seed=43) * NORMS[:, None]
    return tdks, cfg, m, ctx, v, psi


@pytest.mark.parametrize("prec_name", ["fp64", "df64", "mixed", "fp32"])
@pytest.mark.parametrize("kmax", [64, 6])
def test_expm_device_loop_equals_host_loop(prec_name, kmax):
    tdks, cfg, m, ctx, v, psi = _setup()
    prec = {"fp64": tdks.FP64, "df64": tdks.DF64, "mixed": tdks.MIXED, "fp32": tdks.FP32}[prec_name]
    ctx.set_potential(torch.from_numpy(v).cuda())
    if prec_name == "mixed":
        ctx.set_mixed(1e5)
    g = torch.from_numpy(psi).cuda()
    res = {}
    for loop in (0, 1, 1):       # the first device-loop call also fits the captured length
        ctx.set_device_loop(loop)
        ctx.get_counters(reset=True)
        out, k = ctx.expm(g, 0.05, tol=1e-10, k_max=kmax, prec=prec)
        res[loop] = (out.clone(), k, ctx.get_counters())
    assert res[0][1] == res[1][1]
    assert torch.equal(res[0][0], res[1][0])
    c0, c1 = res[0][2], res[1][2]
    assert c0["apply_elem_orb"] == c1["apply_elem_orb"]
    assert c0["apply_launches"] == c1["apply_launches"]
    assert c0["apply_launches_fp32"] == c1["apply_launches_fp32"]
    # host loop: one read per iteration and sub-step; device loop: two per sub-step
    n_sub = max(1, -(-max(res[1][1]) // kmax))
    assert c1["state_reads"] <= 2 * (n_sub + 2) < c0["state_reads"]
    if kmax == 6:
        assert max(res[1][1]) > 6                 # sub-steps were taken
    ctx.close()


def test_expm_device_loop_with_reorthogonalization_and_projectors():
    tdks, cfg, m, ctx, v, psi = _setup(tile=0)
    ctx.set_potential(torch.from_numpy(v).cuda())
    kp = synth.KBParams()
    ctx.set_kb(cfg.atom_R, kp.a, kp.b, kp.c, kp.lmax)
    g = torch.from_numpy(psi).cuda()
    for reorth in (False, True):
        ctx.set_lanczos(reorth)
        outs = []
        for loop in (0, 1):
            ctx.set_device_loop(loop)
            out, k = ctx.expm(g, 0.1, tol=1e-10, k_max=64, prec=tdks.FP64)
            outs.append((out.clone(), k))
        assert outs[0][1] == outs[1][1] and torch.equal(outs[0][0], outs[1][0])
    ctx.close()


@pytest.mark.parametrize("prec_name", ["fp64", "mixed"])
def test_magnus_steps_device_loop_equal_host_loop(prec_name):
    tdks, cfg, m, _, _, _ = _setup()
    prec = {"fp64": tdks.FP64, "mixed": tdks.MIXED}[prec_name]
    psi0 = kick(m, synth.smooth_orbitals(tuple(m.Ni), 6, seed=44) * NORMS[:, None], 0.05, (0.3, -0.5, 0.8))
    runs = {}
    for loop in (0, 1):
        ctx = tdks.Context.from_config(cfg)
        ctx.set_cg(1e-13)
        ctx.set_device_loop(loop)
        ctx.set_timing(True)
        g = torch.from_numpy(psi0).cuda()
        ctx.init_propagation(g)
        step = lambda: ctx.magnus_step(g, 0.1, E_quarter=(0, 0, 0.01), E_half=(0, 0, 0.02), tol=1e-10,
                                       k_max=64, prec=prec)
        step()                   # warm-up: the device loop fits its captured length here
        ctx.get_counters(reset=True)
        st = [step() for _ in range(3)]
        runs[loop] = (g.cpu().numpy(), np.array([s["dipole"] for s in st]), ctx.get_counters(), st)
        ctx.close()
    assert np.array_equal(runs[0][0], runs[1][0]) and np.array_equal(runs[0][1], runs[1][1])
    c0, c1 = runs[0][2], runs[1][2]
    iters = sum(s["k_half_max"] + s["k_full_max"] for s in runs[1][3])
    assert c0["state_reads"] >= iters and c1["state_reads"] <= 3 * 4
    # the device loop times the applications with %globaltimer stamps, the host loop with
    # CUDA events: both see the same work
    assert c1["apply_ms"] > 0 and 0.5 < c1["apply_ms"] / c0["apply_ms"] < 2.0
