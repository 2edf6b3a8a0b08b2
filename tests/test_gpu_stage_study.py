"""Per-stage precision study of the double-float element kernel (tdks_set_f32_stages).

With no stage selected the study switch must leave the double-float application
untouched (bit for bit); with every stage in FP32 the application must carry an error
of the FP32 kernel's size; each single stage must lie between.  The FP64 and FP32
paths ignore the switch, and degrees outside the study's instantiations are refused.
Reference: the oracle's FP64 Hbar application (Eqs. 15, 21; Sec. VI.A).
"""
import numpy as np
import pytest

import synth
from oracle import hamiltonian as ham
from oracle.mesh import Mesh

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


def _setup(p):
    from paper_1810_13130_gb300 import tdks
    cfg = synth.small_config(3, 2, 2, p=p, n_orb=3, seed=23)
    m = Mesh.from_config(cfg)
    ctx = tdks.Context.from_config(cfg)
    v = synth.random_potential(m.n_elem * m.nq ** 3, seed=24).reshape(m.n_elem, -1)
    psi = synth.smooth_orbitals(tuple(m.Ni), 3, seed=25)
    ctx.set_potential(torch.from_numpy(v).cuda())
    return tdks, ctx, torch.from_numpy(psi).cuda(), ham.apply_H(m, v, psi)


@pytest.mark.parametrize("p", [4, 6])
def test_stage_switch_brackets_double_float_and_fp32(p):
    tdks, ctx, g, ref = _setup(p)
    base = ctx.apply_H(g, None, tdks.DF64).cpu().numpy()
    ctx.set_f32_stages(0)
    assert np.array_equal(ctx.apply_H(g, None, tdks.DF64).cpu().numpy(), base)
    e_df = _rel(base, ref)
    e_f32 = _rel(ctx.apply_H(g, None, tdks.FP32).cpu().numpy(), ref)
    ctx.set_f32_stages(0xfff)
    e_all = _rel(ctx.apply_H(g, None, tdks.DF64).cpu().numpy(), ref)
    assert e_df < 1e-12 and 1e-9 < e_f32 < 1e-4
    assert e_f32 / 10 < e_all < e_f32 * 10
    for bit in range(12):
        ctx.set_f32_stages(1 << bit)
        e = _rel(ctx.apply_H(g, None, tdks.DF64).cpu().numpy(), ref)
        assert 10 * e_df < e < 10 * e_all, (bit, e, e_df, e_all)
    # FP64 and FP32 applications ignore the switch
    ctx.set_f32_stages(0x7)
    f64 = ctx.apply_H(g, None, tdks.FP64).cpu().numpy()
    ctx.set_f32_stages(0)
    assert np.array_equal(ctx.apply_H(g, None, tdks.FP64).cpu().numpy(), f64)
    ctx.close()


def test_stage_switch_refuses_other_degrees():
    tdks, ctx, g, _ = _setup(3)
    ctx.set_f32_stages(1)
    with pytest.raises(tdks.TDKSError):
        ctx.apply_H(g, None, tdks.DF64)
    with pytest.raises(tdks.TDKSError):
        ctx.set_f32_stages(1 << 12)
    ctx.close()
