"""Variants on the GPU against the oracle: the self-consistent midpoint step and the
absorption spectrum of a kicked dipole series."""
import numpy as np
import pytest

import synth
from oracle import spectrum
from oracle.mesh import Mesh
from oracle.propagate import Propagator

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


@pytest.mark.parametrize("hartree", [True, False])
def test_self_consistent_midpoint_matches_oracle(hartree):
    from paper_1810_13130_gb300 import tdks
    cfg = synth.small_config(3, 2, 2, p=3, n_orb=2, hartree=hartree)
    m = Mesh.from_config(cfg)
    psi0 = synth.smooth_orbitals(tuple(m.Ni), 2, seed=4)
    prop = Propagator.from_config(cfg, m, tol=1e-12)
    prop.init(psi0)
    ctx = tdks.Context.from_config(cfg)
    ctx.set_cg(1e-13)
    g = torch.from_numpy(psi0).cuda()
    ctx.init_propagation(g)
    ref = psi0
    E = lambda t: np.array([0.02 * np.sin(t), 0.0, 0.01])
    for n in range(3):
        eh = E(n * 0.1 + 0.05)
        ref, dref, it = prop.magnus_step_sc(ref, 0.1, eh, sc_tol=1e-11)
        st = ctx.magnus_step_sc(g, 0.1, eh, tol=1e-12, sc_tol=1e-11)
        assert st["iterations"] == it
        assert _rel(g.cpu().numpy(), ref) < 1e-10
        np.testing.assert_allclose(st["dipole"], dref, rtol=1e-9, atol=1e-12)


def test_self_consistent_midpoint_double_float_matches_oracle():
    """The self-consistent step with double-float contractions: same orbitals as the
    oracle's FP64 iteration to 1e-10 (the iteration count may differ by one at the
    sc_tol boundary)."""
    from paper_1810_13130_gb300 import tdks
    cfg = synth.small_config(3, 2, 2, p=3, n_orb=2, hartree=True)
    m = Mesh.from_config(cfg)
    psi0 = synth.smooth_orbitals(tuple(m.Ni), 2, seed=4)
    prop = Propagator.from_config(cfg, m, tol=1e-12)
    prop.init(psi0)
    ctx = tdks.Context.from_config(cfg)
    ctx.set_cg(1e-13)
    g = torch.from_numpy(psi0).cuda()
    ctx.init_propagation(g)
    ref = psi0
    for n in range(3):
        eh = np.array([0.02 * np.sin(n * 0.1 + 0.05), 0.0, 0.01])
        ref, dref, it = prop.magnus_step_sc(ref, 0.1, eh, sc_tol=1e-11)
        st = ctx.magnus_step_sc(g, 0.1, eh, tol=1e-12, sc_tol=1e-11, prec=tdks.DF64)
        assert abs(st["iterations"] - it) <= 1
        assert _rel(g.cpu().numpy(), ref) < 1e-10
        np.testing.assert_allclose(st["dipole"], dref, rtol=1e-9, atol=1e-12)


def test_self_consistent_midpoint_reports_the_cap():
    from paper_1810_13130_gb300 import tdks
    cfg = synth.small_config(2, 2, 2, p=3, n_orb=1)
    m = Mesh.from_config(cfg)
    ctx = tdks.Context.from_config(cfg)
    g = torch.from_numpy(synth.smooth_orbitals(tuple(m.Ni), 1, seed=2)).cuda()
    ctx.init_propagation(g)
    with pytest.raises(tdks.TDKSError):
        ctx.magnus_step_sc(g, 0.1, sc_tol=1e-30, sc_maxit=2)


def test_spectrum_matches_oracle():
    from paper_1810_13130_gb300 import tdks
    rng = np.random.default_rng(3)
    n, dt, kappa, win = 800, 0.05, 1e-3, 0.005
    t = dt * np.arange(n + 1)
    d = np.zeros((n + 1, 3)) + rng.uniform(-1, 1, 3)
    for w0, amp in ((0.31, 1.0), (0.57, 0.4), (0.9, 0.2)):
        d -= kappa * amp * np.outer(np.sin(w0 * t), rng.uniform(-1, 1, 3))
    om = np.linspace(0.05, 1.2, 64)
    direction = np.array([0.3, -0.5, 0.8])
    a, S = tdks.spectrum(d, dt, kappa, direction, win, om)
    ref_a = spectrum.polarizability(spectrum.windowed(d, win, dt), dt, kappa, direction, om)
    ref_S = spectrum.strength([(d, direction)], dt, kappa, win, om)
    assert _rel(a, ref_a) < 1e-12
    assert _rel(S, ref_S) < 1e-12


@pytest.mark.parametrize("p,n", [(1, (3, 2, 2)), (2, (2, 3, 2)), (4, (2, 2, 3)), (6, (2, 2, 1)), (8, (2, 1, 2))])
def test_gll_collocation_apply_matches_oracle(p, n):
    from oracle import collocation as col
    from paper_1810_13130_gb300 import tdks
    cfg = synth.small_config(*n, p=p, n_orb=2, graded=True)
    m = Mesh.from_config(cfg)
    ctx = tdks.Context.from_config(cfg)
    v = synth.random_potential(m.N_int, 9)
    psi = synth.random_psi(2, m.N_int, 10)
    out = ctx.apply_H_gll(torch.from_numpy(psi).cuda(), torch.from_numpy(v).cuda())
    assert _rel(out.cpu().numpy(), col.apply_H_gll(m, v, psi)) < 1e-12


def test_nuclear_potential_at_nodes():
    from paper_1810_13130_gb300 import tdks
    cfg = synth.small_config(3, 2, 2, p=4, n_orb=1)
    m = Mesh.from_config(cfg)
    ctx = tdks.Context.from_config(cfg)
    X = m.node_coords()
    R = np.asarray(cfg.atom_R)[0]
    ref = -cfg.atom_Z[0] / np.sqrt(np.sum((X - R) ** 2, axis=1) + cfg.nuc_param)
    got = ctx.nuclear_potential_nodes().cpu().numpy()
    np.testing.assert_allclose(got, ref, rtol=1e-14, atol=1e-14)
