"""GPU vs oracle at the launch shapes the benchmark runs: several orbitals per
element-kernel CTA, orbitals leaving the Lanczos recurrence at different j.

The molecule benchmark runs the element kernel with 8 orbitals per CTA (16
orbitals, 820 element blocks): each CTA applies Hbar to its elements for 8
orbitals in turn, skips the orbitals that have converged, accumulates the fused
alpha partials per orbital, and (double-float) prefetches the next active
orbital's input while it computes the current one.  tdks_set_apply_tile forces
that shape on meshes the oracle handles in seconds: 8 orbitals in one CTA
chunk, and 3 (ragged chunks 3, 3, 2).  Compared element by element with the
oracle (Eqs. 36-38 for the exponential; Eqs. 25-26 and Sec. VI.B for the step):
<= 1e-10 relative, Krylov dimensions equal.
"""
import numpy as np
import pytest

import synth
from oracle import hamiltonian as ham
from oracle.lanczos import expm_lanczos
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


def _cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


# Norms spanning six decades: the stopping rule is absolute (Eq. 38 with
# ||psi||), so small orbitals leave the recurrence many iterations earlier.
NORMS = np.array([1.0, 1e-3, 1.0, 1e-6, 0.3, 1.0, 1e-2, 1.0])


def _system():
    cfg = synth.small_config(3, 3, 2, p=6, n_orb=8, graded=True, seed=31)
    return cfg, Mesh.from_config(cfg)


def _uneven_block(m, seed):
    """Smooth and rough orbitals interleaved, with unequal norms."""
    smooth = synth.smooth_orbitals(tuple(m.Ni), 4, seed=seed)
    rough = synth.random_psi(4, m.N_int, seed=seed + 1)
    psi = np.empty((8, m.N_int), complex)
    psi[0::2] = smooth
    psi[1::2] = rough
    return psi * NORMS[:, None]


TAU = 0.05
E_Q, E_H = (0.0, 0.0, 0.01), (0.0, 0.0, 0.02)


@pytest.fixture(scope="module")
def expm_ref():
    cfg, m = _system()
    v = synth.random_potential(m.n_elem * m.nq ** 3, seed=33).reshape(m.n_elem, -1)
    psi = _uneven_block(m, 34)
    ref, info = expm_lanczos(lambda x: ham.apply_H(m, v, x), psi, TAU, 1e-10, 64)
    return cfg, m, v, psi, ref, [sum(ks) for ks in info["k"]]


@pytest.fixture(scope="module")
def step_ref():
    cfg, m = _system()
    psi0 = kick(m, synth.smooth_orbitals(tuple(m.Ni), 8, seed=35) * NORMS[:, None], 0.05,
                (0.3, -0.5, 0.8))
    prop = Propagator.from_config(cfg, m, cg_tol=1e-13)
    d0 = prop.init(psi0)
    ref, dref, info = prop.magnus_step(psi0, 0.1, E_quarter=E_Q, E_half=E_H)
    kh = [sum(k) for k in info["k_half"]]
    kf = [sum(k) for k in info["k_full"]]
    return cfg, m, psi0, d0, ref, dref, kh, kf


@pytest.mark.parametrize("tile", [8, 3])
@pytest.mark.parametrize("prec_name", ["fp64", "df64"])
def test_expm_multi_orbital_cta_matches_oracle(tile, prec_name, expm_ref):
    from paper_1810_13130_gb300 import tdks
    prec = {"fp64": tdks.FP64, "df64": tdks.DF64}[prec_name]
    cfg, m, v, psi, ref, k_ref = expm_ref
    ctx = tdks.Context.from_config(cfg)
    ctx.set_apply_tile(tile)
    ctx.set_potential(_cuda(v))
    out, k = ctx.expm(_cuda(psi), TAU, tol=1e-10, k_max=64, prec=prec)
    assert max(k_ref) - min(k_ref) >= 4          # orbitals leave the recurrence unevenly
    if prec_name == "df64" and k != k_ref:
        # a double-float alpha/beta may move a stopping decision that sits at the
        # tolerance by one: replay the oracle at the GPU's dimensions
        assert all(abs(a - b) <= 1 for a, b in zip(k, k_ref)) and max(k) <= 64
        ref, _ = expm_lanczos(lambda x: ham.apply_H(m, v, x), psi, TAU, 1e-10, 64, k_fixed=k)
    else:
        assert k == k_ref
    assert _rel(out.cpu().numpy(), ref) < 1e-10
    ctx.close()


@pytest.mark.parametrize("tile", [8, 3])
@pytest.mark.parametrize("prec_name", ["fp64", "df64"])
def test_magnus_step_multi_orbital_cta_matches_oracle(tile, prec_name, step_ref):
    from paper_1810_13130_gb300 import tdks
    prec = {"fp64": tdks.FP64, "df64": tdks.DF64}[prec_name]
    cfg, m, psi0, d0, ref, dref, kh, kf = step_ref
    ctx = tdks.Context.from_config(cfg)
    ctx.set_cg(1e-13)
    ctx.set_apply_tile(tile)
    g = _cuda(psi0)
    dg0 = ctx.init_propagation(g)
    st = ctx.magnus_step(g, 0.1, E_quarter=E_Q, E_half=E_H, tol=1e-10, k_max=64, prec=prec)
    assert max(kf) - min(kf) >= 4                 # uneven convergence across the CTA's orbitals
    assert st["k_half_max"] == max(kh) and st["k_full_max"] == max(kf)
    assert _rel(g.cpu().numpy(), ref) < 1e-10
    assert _rel(dg0, d0) < 1e-12 and _rel(st["dipole"], dref) < 1e-10
    ctx.close()


def test_apply_tile_does_not_change_results():
    """Hbar psi is identical (bit for bit) for every tile, in FP64 and double-float:
    each orbital's arithmetic does not depend on which CTA chunk it falls in."""
    from paper_1810_13130_gb300 import tdks
    cfg, m = _system()
    ctx = tdks.Context.from_config(cfg)
    v = synth.random_potential(m.n_elem * m.nq ** 3, seed=36).reshape(m.n_elem, -1)
    ctx.set_potential(_cuda(v))
    psi = _cuda(_uneven_block(m, 37))
    outs = []
    for tile in (0, 1, 2, 3, 5, 8, 64):
        ctx.set_apply_tile(tile)
        outs.append([ctx.apply_H(psi, prec=p).cpu().numpy() for p in (tdks.FP64, tdks.DF64)])
    for o in outs[1:]:
        assert np.array_equal(o[0], outs[0][0]) and np.array_equal(o[1], outs[0][1])
    with pytest.raises(tdks.TDKSError):
        ctx.set_apply_tile(-1)
    ctx.close()


@pytest.mark.parametrize("tile", [8, 3])
def test_expm_relaxed_precision_matches_oracle(tile, expm_ref):
    """TDKS_MIXED: double-float products until every active orbital's estimate of Eq. 38
    is below relax * tol, FP32 products after.  The stopping rule is unchanged, so the
    Krylov dimensions stay within one of the oracle's and the result within a few
    tolerances; the FP32 share must be non-zero for the schedule to be exercised."""
    from paper_1810_13130_gb300 import tdks
    cfg, m, v, psi, ref, k_ref = expm_ref
    ctx = tdks.Context.from_config(cfg)
    ctx.set_apply_tile(tile)
    ctx.set_potential(_cuda(v))
    # a switch level of 1e5 x tol: the FP32 products add far less than the tolerance
    ctx.set_mixed(1e5)
    ctx.get_counters(reset=True)
    out, k = ctx.expm(_cuda(psi), TAU, tol=1e-10, k_max=64, prec=tdks.MIXED)
    cnt = ctx.get_counters()
    assert 0 < cnt["apply_launches_fp32"] < cnt["apply_launches"]
    assert all(abs(a - b) <= 1 for a, b in zip(k, k_ref))
    err = np.abs(out.cpu().numpy() - ref).max(axis=1)
    assert err.max() < 1e-9, err
    # the default level (1e8 x tol): FP32 products once every estimate is <= 1e-2;
    # each adds about 1e-6 of its estimate, so the exponential stays within 1e-7
    ctx.set_mixed(1e8)
    ctx.get_counters(reset=True)
    out, k = ctx.expm(_cuda(psi), TAU, tol=1e-10, k_max=64, prec=tdks.MIXED)
    cnt = ctx.get_counters()
    assert cnt["apply_launches_fp32"] > 0
    assert np.abs(out.cpu().numpy() - ref).max() < 1e-7
    ctx.set_mixed(0.0)                     # never relaxed: the double-float path
    out_df, _ = ctx.expm(_cuda(psi), TAU, tol=1e-10, k_max=64, prec=tdks.MIXED)
    ref_df, _ = ctx.expm(_cuda(psi), TAU, tol=1e-10, k_max=64, prec=tdks.DF64)
    assert torch.equal(out_df, ref_df)
    ctx.close()
