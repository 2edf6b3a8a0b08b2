"""Nonlocal Kleinman-Bylander term (Eq. 6, Galerkin and Loewdin form) on the GPU against
the oracle: denominators, the Hbar application with the term, the Lanczos exponential,
Magnus steps and the adjoint gradient with projectors present."""
import numpy as np
import pytest

import synth
from oracle import adjoint
from oracle import hamiltonian as ham
from oracle.kb import KleinmanBylander
from oracle.lanczos import expm_lanczos
from oracle.mesh import Mesh
from oracle.propagate import Propagator

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ATOMS = np.array([[0.3, -0.2, 0.1], [-2.1, 1.4, 0.9]])


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1810_13130_gb300.build import build
    build()


def _rel(a, b):
    return float(np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(b).max(), 1e-300))


def _setup(p, n=(3, 2, 2), lmax=1):
    from paper_1810_13130_gb300 import tdks
    cfg = synth.small_config(*n, p=p, n_orb=2)
    m = Mesh.from_config(cfg)
    kp = synth.KBParams(lmax=lmax)
    kb = KleinmanBylander(m, ATOMS, kp.a, kp.b, kp.c, lmax=kp.lmax)
    ctx = tdks.Context.from_config(cfg)
    ctx.set_cg(1e-13)
    ctx.set_kb(ATOMS, kp.a, kp.b, kp.c, kp.lmax)
    return cfg, m, kb, ctx


@pytest.mark.parametrize("p,lmax", [(2, 1), (3, 0), (5, 1), (8, 1)])
def test_apply_with_projectors_matches_oracle(p, lmax):
    cfg, m, kb, ctx = _setup(p, (2, 2, 2) if p == 8 else (3, 2, 2), lmax)
    info = ctx.kb_info()
    np.testing.assert_allclose(info["h"], kb.h, rtol=1e-12)
    v = synth.random_potential(m.n_elem * m.nq ** 3, 5).reshape(m.n_elem, -1)
    psi = synth.random_psi(2, m.N_int, 3)
    ctx.set_potential(torch.from_numpy(v).cuda())
    out = ctx.apply_H(torch.from_numpy(psi).cuda())
    ref = ham.apply_H(m, v, psi) + kb.apply(psi)
    assert _rel(out.cpu().numpy(), ref) < 1e-12


def test_removing_the_projectors_restores_the_local_operator():
    cfg, m, kb, ctx = _setup(3)
    v = synth.random_potential(m.n_elem * m.nq ** 3, 6).reshape(m.n_elem, -1)
    psi = synth.random_psi(2, m.N_int, 4)
    ctx.set_potential(torch.from_numpy(v).cuda())
    ctx.set_kb(np.zeros((0, 3)))
    assert ctx.kb_info()["n_proj"] == 0
    out = ctx.apply_H(torch.from_numpy(psi).cuda())
    assert _rel(out.cpu().numpy(), ham.apply_H(m, v, psi)) < 1e-12


def test_expm_with_projectors_matches_oracle():
    cfg, m, kb, ctx = _setup(4)
    v = synth.random_potential(m.n_elem * m.nq ** 3, 7).reshape(m.n_elem, -1)
    psi = synth.random_psi(2, m.N_int, 8)
    ctx.set_potential(torch.from_numpy(v).cuda())
    out, k = ctx.expm(torch.from_numpy(psi).cuda(), 0.2, tol=1e-12, k_max=64)
    ref, info = expm_lanczos(lambda x: ham.apply_H(m, v, x) + kb.apply(x), psi, 0.2, 1e-12, 64)
    assert k == [sum(x) for x in info["k"]]
    assert _rel(out.cpu().numpy(), ref) < 1e-10


@pytest.mark.parametrize("prec", ["fp64", "df64"])
def test_magnus_steps_with_projectors_match_oracle(prec):
    """Local contractions in FP64 or double-float; the projector term is FP64 in both."""
    from paper_1810_13130_gb300 import tdks
    pr = {"fp64": tdks.FP64, "df64": tdks.DF64}[prec]
    cfg, m, kb, ctx = _setup(3)
    psi0 = synth.smooth_orbitals(tuple(m.Ni), 2, seed=4)
    prop = Propagator.from_config(cfg, m, nl=kb)
    prop.init(psi0)
    g = torch.from_numpy(psi0).cuda()
    ctx.init_propagation(g)
    ref = psi0
    for n in range(3):
        ref, dref, _ = prop.magnus_step(ref, cfg.dt)
        st = ctx.magnus_step(g, cfg.dt, prec=pr)
        assert _rel(g.cpu().numpy(), ref) < 1e-10
        np.testing.assert_allclose(st["dipole"], dref, rtol=1e-9, atol=1e-12)


def test_adjoint_with_projectors_matches_oracle():
    cfg, m, kb, ctx = _setup(3)
    psi0 = synth.smooth_orbitals(tuple(m.Ni), 2, seed=5)
    N, dt = 3, 0.1
    rng = np.random.default_rng(6)
    E = rng.uniform(-0.05, 0.05, size=(N, 2, 3))
    w = np.full(N + 1, dt)
    w[0] = w[-1] = 0.5 * dt
    e = np.array([0.2, -0.3, 0.93])
    prop = Propagator.from_config(cfg, m, tol=1e-12, k_max=200, nl=kb)
    J_o, g_o = adjoint.objective_and_gradient(prop, psi0, E, w, e, dt, n_s=12, tol_adj=1e-12)
    J, _ = ctx.objective_forward(torch.from_numpy(psi0).cuda(), E.reshape(-1, 6), w, e, dt,
                                 ckpt_every=2, tol=1e-12, k_max=64)
    g = ctx.objective_backward(n_s=12)
    assert abs(J - J_o) <= 1e-10 * abs(J_o)
    assert np.abs(g - g_o.reshape(-1, 6)).max() <= 1e-8 * np.abs(g_o).max()
