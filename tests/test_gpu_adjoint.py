"""GPU adjoint of the Magnus predictor-corrector propagation (C-ABI) against the
oracle's FP64 adjoint and against central finite differences of the GPU forward.

Objective J = sum_n w_n (e . mu_n)^2 (dipole response, Sec. V) as a function of the
field samples of Sec. VI.B; the pulse test differentiates through torch.autograd
down to the parameters of four Gaussian-envelope pulses.
"""
import os

import numpy as np
import pytest

import synth
from oracle import adjoint
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


def _ctx(cfg):
    from paper_1810_13130_gb300 import tdks
    c = tdks.Context.from_config(cfg)
    c.set_cg(1e-13)
    return c


def _small_problem(hartree, n_steps=5, seed=6):
    cfg = synth.small_config(3, 2, 2, p=3, n_orb=2, hartree=hartree)
    m = Mesh.from_config(cfg)
    psi0 = synth.smooth_orbitals(tuple(m.Ni), 2, seed=5)
    rng = np.random.default_rng(seed)
    E = rng.uniform(-0.05, 0.05, size=(n_steps, 2, 3))
    dt = 0.1
    w = np.full(n_steps + 1, dt)
    w[0] = w[-1] = 0.5 * dt
    e = np.array([0.2, -0.3, 0.93])
    return cfg, m, psi0, E, w, e, dt


@pytest.mark.parametrize("hartree", [True, False])
def test_adjoint_matches_oracle_small_system(hartree):
    cfg, m, psi0, E, w, e, dt = _small_problem(hartree)
    prop = Propagator.from_config(cfg, m, tol=1e-12, k_max=200)
    J_o, g_o = adjoint.objective_and_gradient(prop, psi0, E, w, e, dt, n_s=12, tol_adj=1e-12)
    ctx = _ctx(cfg)
    psi = torch.from_numpy(psi0).cuda()
    J, dip = ctx.objective_forward(psi, E.reshape(-1, 6), w, e, dt, ckpt_every=2, tol=1e-12,
                                   k_max=64)
    g = ctx.objective_backward(n_s=12)
    assert abs(J - J_o) <= 1e-10 * abs(J_o)
    assert np.abs(g - g_o.reshape(-1, 6)).max() <= 1e-8 * np.abs(g_o).max()
    # psi0 is untouched by the forward call
    assert torch.equal(psi.cpu(), torch.from_numpy(psi0))


def test_adjoint_with_double_float_forward_matches_oracle():
    """The objective propagated with double-float contractions (recomputed the same way
    in the backward sweep): J and the gradient against the oracle's FP64 adjoint."""
    from paper_1810_13130_gb300 import tdks
    cfg, m, psi0, E, w, e, dt = _small_problem(True)
    prop = Propagator.from_config(cfg, m, tol=1e-12, k_max=200)
    J_o, g_o = adjoint.objective_and_gradient(prop, psi0, E, w, e, dt, n_s=12, tol_adj=1e-12)
    ctx = _ctx(cfg)
    psi = torch.from_numpy(psi0).cuda()
    J, _ = ctx.objective_forward(psi, E.reshape(-1, 6), w, e, dt, ckpt_every=2, tol=1e-12,
                                 k_max=64, prec=tdks.DF64)
    g = ctx.objective_backward(n_s=12)
    assert abs(J - J_o) <= 1e-10 * abs(J_o)
    assert np.abs(g - g_o.reshape(-1, 6)).max() <= 1e-8 * np.abs(g_o).max()


def test_adjoint_checkpoint_interval_does_not_change_the_result():
    """Recomputation from a checkpoint replays the forward bit for bit (every kernel
    reduces in a fixed order), so the gradient cannot depend on the interval."""
    cfg, m, psi0, E, w, e, dt = _small_problem(True, n_steps=6, seed=9)
    ctx = _ctx(cfg)
    psi = torch.from_numpy(psi0).cuda()
    out = []
    for K in (1, 4, 6):
        J, _ = ctx.objective_forward(psi, E.reshape(-1, 6), w, e, dt, ckpt_every=K, tol=1e-12,
                                     k_max=64)
        out.append((J, ctx.objective_backward(n_s=8)))
    for J, g in out[1:]:
        assert J == out[0][0]
        np.testing.assert_array_equal(g, out[0][1])


def test_adjoint_rejects_bad_calls():
    from paper_1810_13130_gb300 import tdks
    cfg, m, psi0, E, w, e, dt = _small_problem(False, n_steps=2)
    ctx = _ctx(cfg)
    with pytest.raises(tdks.TDKSError):
        ctx.objective_backward(8)                 # no forward yet
    psi = torch.from_numpy(psi0).cuda()
    ctx.objective_forward(psi, E.reshape(-1, 6), w, e, dt, ckpt_every=1, tol=1e-12)
    with pytest.raises(tdks.TDKSError):
        ctx.objective_backward(0)
    with pytest.raises(tdks.TDKSError):
        ctx.objective_forward(psi, E.reshape(-1, 6), w[:-1], e, dt)


def _atom_ground_state(cfg):
    gs = np.load(os.path.join(os.path.dirname(__file__), "golden", "gs_atom_soft_Z2_6x6x6_p4.npz"))
    return gs["psibar"].astype(complex)


def test_pulse_parameter_gradient_matches_central_differences():
    """The atom driven by four Gaussian pulses, 200 steps of dt = 0.1, checkpoints every
    20 steps: d/d(a_j, phi_j) of int d_z(t)^2 dt, adjoint vs central differences
    (h = 1e-5) of the GPU forward, <= 1e-5 relative."""
    from paper_1810_13130_gb300 import tdks
    sc, pc = synth.config4()
    ctx = _ctx(sc)
    psi0 = torch.from_numpy(_atom_ground_state(sc)).cuda()
    w = pc.objective_weights()
    e = np.asarray(pc.direction)
    tol, kmax = 1e-12, 64

    params = torch.tensor(pc.params, dtype=torch.float64, requires_grad=True)
    E = synth.pulse_samples(params, pc)
    J = tdks.DipoleObjective.apply(E, ctx, psi0, w, e, pc.dt, pc.ckpt_every, tol, kmax,
                                   tdks.FP64, 12)
    J.backward()
    g = params.grad.numpy().copy()
    assert J.item() > 0

    def J_of(p):
        Ep = synth.pulse_samples(p, pc)
        return ctx.objective_forward(psi0, Ep, w, e, pc.dt, pc.ckpt_every, tol, kmax)[0]

    h = pc.fd_h
    fd = np.zeros_like(g)
    base = pc.params
    for k in range(len(base)):
        pp, pm = base.copy(), base.copy()
        pp[k] += h
        pm[k] -= h
        fd[k] = (J_of(pp) - J_of(pm)) / (2 * h)
    rel = np.abs(g - fd) / np.abs(fd).max()
    assert rel.max() <= 1e-5, (g, fd, rel)
