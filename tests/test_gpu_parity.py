"""GPU (C-ABI) vs CPU oracle parity, element by element on seeded inputs.

Tolerances: FP64 operators (apply_H, density, XC, V_N, dipole) agree to
rounding, <= 1e-12 relative to the largest entry; the Lanczos exponential,
Poisson solve and Magnus step agree to <= 1e-10 relative (the orbital
tolerance of the FP64 path); FP32 contractions are reported against the FP64
oracle with a 1e-5 bound.
"""
import numpy as np
import pytest

import synth
from oracle import hamiltonian as ham
from oracle import poisson, xc
from oracle.lanczos import expm_lanczos
from oracle.mesh import Mesh
from oracle.propagate import Propagator, kick, nuclear_potential

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


def _rel(a, b):
    return float(np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(b).max(), 1e-300))


def _cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


SMALL = [(1, (3, 2, 2)), (2, (3, 2, 3)), (3, (3, 2, 2)), (4, (2, 3, 2)), (5, (2, 2, 3)),
         (6, (3, 2, 1)), (7, (2, 1, 2)), (8, (2, 2, 1))]


@pytest.mark.parametrize("p,n", SMALL)
def test_apply_H_fp64_every_degree(p, n):
    cfg = synth.small_config(*n, p=p, n_orb=3, graded=(p % 2 == 0))
    m = Mesh.from_config(cfg)
    ctx = _ctx(cfg)
    psi = synth.random_psi(3, m.N_int, seed=100 + p)
    v = synth.random_potential(m.n_elem * m.nq ** 3, seed=200 + p).reshape(m.n_elem, -1)
    ctx.set_potential(_cuda(v))
    got = ctx.apply_H(_cuda(psi)).cpu().numpy()
    assert _rel(got, ham.apply_H(m, v, psi)) < 1e-12


def test_apply_H_fp64_atom_workload_full():
    cfg = synth.config1()
    m = Mesh.from_config(cfg)
    ctx = _ctx(cfg)
    psi = synth.random_psi(1, m.N_int, seed=5)
    v = synth.random_potential(m.n_elem * m.nq ** 3, seed=6).reshape(m.n_elem, -1)
    ctx.set_potential(_cuda(v))
    got = ctx.apply_H(_cuda(psi)).cpu().numpy()
    assert _rel(got, ham.apply_H(m, v, psi)) < 1e-12


def test_apply_H_molecule_workload_sampled_rows():
    """16^3 elements, p = 6, 16 orbitals (the benchmarked size): sampled outputs."""
    cfg = synth.config2()
    m = Mesh.from_config(cfg)
    ctx = _ctx(cfg)
    psi = synth.random_psi(cfg.n_orb, m.N_int, seed=7)
    v = synth.random_potential(m.n_elem * m.nq ** 3, seed=8).reshape(m.n_elem, -1)
    ctx.set_potential(_cuda(v))
    got = ctx.apply_H(_cuda(psi)).cpu().numpy()
    rng = np.random.default_rng(9)
    rows = np.concatenate([rng.choice(m.N_int, 40, replace=False), [0, m.N_int - 1, m.Ni[0] - 1]])
    ref = ham.apply_H_rows(m, v, psi, rows)
    assert _rel(got[:, rows], ref) < 1e-12
    # hermiticity at full size: <a, H b> = conj(<b, H a>)
    a, b = _cuda(psi[0:1]), _cuda(psi[1:2])
    Ha, Hb = ctx.apply_H(a), ctx.apply_H(b)
    lhs = torch.vdot(a.flatten(), Hb.flatten()).item()
    rhs = torch.vdot(b.flatten(), Ha.flatten()).item().conjugate()
    assert abs(lhs - rhs) < 1e-11 * abs(Ha).max().item()


def test_apply_H_graded_workload_sampled_rows():
    """Graded 24^3 mesh, p = 8, 5 orbitals (the all-electron-like workload, 6.97 M DoF):
    sampled outputs of the FP64 and double-float contractions against the oracle."""
    from paper_1810_13130_gb300 import tdks
    cfg = synth.config3()
    m = Mesh.from_config(cfg)
    ctx = _ctx(cfg)
    psi = synth.random_psi(cfg.n_orb, m.N_int, seed=11)
    v = synth.random_potential(m.n_elem * m.nq ** 3, seed=12).reshape(m.n_elem, -1)
    ctx.set_potential(_cuda(v))
    g = _cuda(psi)
    got = ctx.apply_H(g).cpu().numpy()
    got_df = ctx.apply_H(g, prec=tdks.DF64).cpu().numpy()
    rng = np.random.default_rng(13)
    rows = np.concatenate([rng.choice(m.N_int, 30, replace=False), [0, m.N_int - 1, m.N_int // 2]])
    ref = ham.apply_H_rows(m, v, psi, rows)
    assert _rel(got[:, rows], ref) < 1e-12
    assert _rel(got_df[:, rows], ref) < 1e-11


def test_apply_H_fp32_error_vs_fp64_oracle():
    cfg = synth.small_config(3, 3, 2, p=6, n_orb=2)
    m = Mesh.from_config(cfg)
    ctx = _ctx(cfg)
    psi = synth.random_psi(2, m.N_int, seed=10)
    v = synth.random_potential(m.n_elem * m.nq ** 3, seed=11).reshape(m.n_elem, -1)
    ctx.set_potential(_cuda(v))
    from paper_1810_13130_gb300 import tdks
    got = ctx.apply_H(_cuda(psi), prec=tdks.FP32).cpu().numpy()
    err = _rel(got, ham.apply_H(m, v, psi))
    assert 1e-9 < err < 1e-5


def test_apply_H_bf16_operand_error_vs_fp64_oracle():
    """BF16-operand mode (bfloat16 operands, FP32 products and sums): an error at the
    bfloat16 level (8-bit significand, ~4e-3 per rounding), far above FP32's."""
    from paper_1810_13130_gb300 import tdks
    cfg = synth.small_config(3, 3, 2, p=6, n_orb=2)
    m = Mesh.from_config(cfg)
    ctx = _ctx(cfg)
    psi = synth.random_psi(2, m.N_int, seed=10)
    v = synth.random_potential(m.n_elem * m.nq ** 3, seed=11).reshape(m.n_elem, -1)
    ctx.set_potential(_cuda(v))
    ref = ham.apply_H(m, v, psi)
    e16 = _rel(ctx.apply_H(_cuda(psi), prec=tdks.BF16).cpu().numpy(), ref)
    e32 = _rel(ctx.apply_H(_cuda(psi), prec=tdks.FP32).cpu().numpy(), ref)
    assert 1e-4 < e16 < 5e-2
    assert e16 > 100 * e32


@pytest.mark.parametrize("p,n", [(3, (3, 2, 2)), (6, (3, 2, 2)), (8, (2, 2, 1))])
def test_apply_H_df64_matches_fp64_oracle(p, n):
    """Double-float contractions: FP64-level agreement (~48-bit arithmetic)."""
    from paper_1810_13130_gb300 import tdks
    cfg = synth.small_config(*n, p=p, n_orb=2, graded=True)
    m = Mesh.from_config(cfg)
    ctx = _ctx(cfg)
    psi = synth.random_psi(2, m.N_int, seed=30 + p)
    v = synth.random_potential(m.n_elem * m.nq ** 3, seed=40 + p).reshape(m.n_elem, -1)
    ctx.set_potential(_cuda(v))
    got = ctx.apply_H(_cuda(psi), prec=tdks.DF64).cpu().numpy()
    assert _rel(got, ham.apply_H(m, v, psi)) < 1e-11


@pytest.mark.parametrize("precond", [0, 1])
def test_fields_match_oracle(precond):
    cfg = synth.small_config(3, 2, 2, p=4, n_orb=2, nuc_kind="erf", graded=True)
    cfg.nuc_param = 0.8
    m = Mesh.from_config(cfg)
    ctx = _ctx(cfg)
    ctx.set_cg(1e-13, 5000, precond)
    vn_ref = nuclear_potential(m, "erf", cfg.atom_R, cfg.atom_Z, 0.8)
    assert _rel(ctx.nuclear_potential().cpu().numpy(), vn_ref) < 1e-14
    psi = synth.smooth_orbitals(tuple(m.Ni), 2, seed=3)
    rho = ctx.density(_cuda(psi))
    rho_ref = ham.density(m, psi, cfg.occ)
    assert _rel(rho.cpu().numpy(), rho_ref) < 1e-12
    np.testing.assert_allclose(ctx.dipole(rho), ham.dipole(m, rho_ref), rtol=1e-12, atol=1e-14)
    assert _rel(ctx.xc(rho).cpu().numpy(), xc.v_xc(rho_ref)) < 1e-13
    vh, it = ctx.hartree(rho)
    vh_ref, _, _ = poisson.hartree(m, rho_ref, tol=1e-13)
    assert _rel(vh.cpu().numpy(), vh_ref) < 1e-10 and it > 0
    if precond == 0:
        assert it <= 3          # exact inverse: one or two iterations
    # warm start: the same right-hand side again converges at once
    vh2, it2 = ctx.hartree(rho)
    assert it2 <= 1 and _rel(vh2.cpu().numpy(), vh_ref) < 1e-10


def test_hartree_molecule_workload_fdm():
    """Full-size Poisson solve: FDM-preconditioned CG agrees with Jacobi CG."""
    cfg = synth.config2()
    m = Mesh.from_config(cfg)
    psi = synth.smooth_orbitals(tuple(m.Ni), cfg.n_orb, seed=1)
    a, b = _ctx(cfg), _ctx(cfg)
    a.set_cg(1e-12, 5000, 0)
    b.set_cg(1e-12, 5000, 1)
    rho = a.density(_cuda(psi))
    va, ia = a.hartree(rho)
    vb, ib = b.hartree(rho)
    assert ia <= 3 < ib
    assert _rel(va.cpu().numpy(), vb.cpu().numpy()) < 1e-9


@pytest.mark.parametrize("kind", ["soft", "bare", "harmonic"])
def test_nuclear_kinds(kind):
    cfg = synth.small_config(2, 3, 2, p=3, n_orb=1, nuc_kind=kind)
    m = Mesh.from_config(cfg)
    ctx = _ctx(cfg)
    ref = nuclear_potential(m, kind, cfg.atom_R, cfg.atom_Z, cfg.nuc_param)
    assert _rel(ctx.nuclear_potential().cpu().numpy(), ref) < 1e-14


@pytest.mark.parametrize("tau,kmax", [(0.05, 64), (0.3, 64), (0.5, 6)])
def test_expm_matches_oracle(tau, kmax):
    cfg = synth.small_config(3, 2, 2, p=4, n_orb=3)
    m = Mesh.from_config(cfg)
    ctx = _ctx(cfg)
    v = synth.random_potential(m.n_elem * m.nq ** 3, seed=21).reshape(m.n_elem, -1)
    ctx.set_potential(_cuda(v))
    psi = synth.random_psi(3, m.N_int, seed=22) * np.array([[1.0], [0.5], [2.0]])
    out, k = ctx.expm(_cuda(psi), tau, tol=1e-10, k_max=kmax)
    ref, info = expm_lanczos(lambda x: ham.apply_H(m, v, x), psi, tau, 1e-10, kmax)
    assert k == [sum(ks) for ks in info["k"]]
    assert _rel(out.cpu().numpy(), ref) < 1e-10
    if kmax == 6:
        assert max(len(ks) for ks in info["k"]) > 1      # sub-steps were exercised


@pytest.mark.parametrize("tau,kmax", [(0.3, 64), (0.5, 6)])
def test_expm_with_reorthogonalization_matches_oracle(tau, kmax):
    """CGS2 re-orthogonalized Lanczos (tdks_set_lanczos) against the oracle's, including
    sub-steps; and against the plain recurrence (same exponential within tolerance)."""
    cfg = synth.small_config(3, 2, 2, p=4, n_orb=3)
    m = Mesh.from_config(cfg)
    ctx = _ctx(cfg)
    v = synth.random_potential(m.n_elem * m.nq ** 3, seed=23).reshape(m.n_elem, -1)
    ctx.set_potential(_cuda(v))
    psi = synth.random_psi(3, m.N_int, seed=24) * np.array([[1.0], [0.5], [2.0]])
    ctx.set_lanczos(True)
    out, k = ctx.expm(_cuda(psi), tau, tol=1e-10, k_max=kmax)
    ref, info = expm_lanczos(lambda x: ham.apply_H(m, v, x), psi, tau, 1e-10, kmax, reorth=True)
    assert k == [sum(ks) for ks in info["k"]]
    assert _rel(out.cpu().numpy(), ref) < 1e-10
    ctx.set_lanczos(False)
    plain, _ = ctx.expm(_cuda(psi), tau, tol=1e-10, k_max=kmax)
    assert _rel(out.cpu().numpy(), plain.cpu().numpy()) < 1e-9


def test_expm_df64_two_orbitals_per_cta_with_uneven_convergence():
    """Double-float Lanczos on a mesh large enough that each element-kernel CTA runs two
    orbitals (3072 elements, p = 6: 615 CTAs per orbital pair), with smooth and rough
    orbitals that leave the recurrence at different j: the CTA skips the converged
    orbital and prefetches the next active one.  Against the FP64 path, which equals
    the oracle on the small systems above."""
    from paper_1810_13130_gb300 import tdks
    cfg = synth.small_config(16, 16, 12, p=6, n_orb=4, L=16.0)
    m = Mesh.from_config(cfg)
    ctx = _ctx(cfg)
    v = synth.random_potential(m.n_elem * m.nq ** 3, seed=25).reshape(m.n_elem, -1)
    ctx.set_potential(_cuda(v))
    smooth = synth.smooth_orbitals(tuple(m.Ni), 2, seed=26)
    rough = synth.random_psi(2, m.N_int, seed=27)
    psi = np.stack([smooth[0], rough[0], smooth[1], rough[1]])
    out64, k64 = ctx.expm(_cuda(psi), 0.1, tol=1e-10, k_max=64)
    outdf, kdf = ctx.expm(_cuda(psi), 0.1, tol=1e-10, k_max=64, prec=tdks.DF64)
    assert min(k64[0], k64[2]) < max(k64[1], k64[3])   # the smooth orbitals leave first
    assert _rel(outdf.cpu().numpy(), out64.cpu().numpy()) < 1e-10
    assert max(abs(a - b) for a, b in zip(kdf, k64)) <= 1


def test_expm_edge_cases():
    from paper_1810_13130_gb300 import tdks
    cfg = synth.small_config(2, 2, 2, p=2, n_orb=2)
    m = Mesh.from_config(cfg)
    ctx = _ctx(cfg)
    z = torch.zeros((2, m.N_int), dtype=torch.complex128, device="cuda")
    out, k = ctx.expm(z, 0.2)
    assert torch.count_nonzero(out).item() == 0
    with pytest.raises(tdks.TDKSError):
        ctx.expm(z, 0.2, k_max=500)
    # an eigenvector of Hbar breaks down at k = 1 with the exact phase
    v = np.zeros((m.n_elem, m.nq ** 3))
    ctx.set_potential(_cuda(v))
    H = ham.dense_Hbar(m, v)
    lam, S = np.linalg.eigh(H)
    e = np.stack([S[:, 0], S[:, 5]]).astype(complex)
    out, k = ctx.expm(_cuda(e), 0.7)
    assert k == [1, 1]
    np.testing.assert_allclose(out.cpu().numpy(), np.exp(-0.7j * lam[[0, 5]])[:, None] * e, atol=1e-12)


@pytest.mark.parametrize("tau,kmax", [(10.0, 128), (0.05, 4), (0.02, 3)])
def test_expm_at_the_krylov_limits_matches_oracle(tau, kmax):
    """Krylov spaces beyond the default cap (72 vectors under the largest cap, 128) and
    tiny caps (3, 4: tens to a hundred sub-steps) against the oracle's Lanczos with the
    same cap."""
    cfg = synth.small_config(3, 2, 2, p=4, n_orb=2)
    m = Mesh.from_config(cfg)
    ctx = _ctx(cfg)
    v = synth.random_potential(m.n_elem * m.nq ** 3, seed=28).reshape(m.n_elem, -1)
    ctx.set_potential(_cuda(v))
    psi = synth.random_psi(2, m.N_int, seed=29)
    out, k = ctx.expm(_cuda(psi), tau, tol=1e-10, k_max=kmax)
    ref, info = expm_lanczos(lambda x: ham.apply_H(m, v, x), psi, tau, 1e-10, kmax)
    assert k == [sum(ks) for ks in info["k"]]
    assert _rel(out.cpu().numpy(), ref) < 1e-10
    if kmax == 128:
        assert min(max(ks) for ks in info["k"]) > 64
    else:
        assert min(len(ks) for ks in info["k"]) > 20          # many sub-steps


def test_bad_orbital_counts_are_rejected():
    from paper_1810_13130_gb300 import tdks
    cfg = synth.small_config(2, 2, 2, p=2, n_orb=2)
    m = Mesh.from_config(cfg)
    ctx = _ctx(cfg)
    three = torch.zeros((3, m.N_int), dtype=torch.complex128, device="cuda")
    empty = torch.zeros((0, m.N_int), dtype=torch.complex128, device="cuda")
    # apply_H takes any number of vectors (>= 1); the Krylov calls are bounded by the
    # system's orbital count
    assert torch.count_nonzero(ctx.apply_H(three)).item() == 0
    with pytest.raises(tdks.TDKSError):
        ctx.apply_H(empty)
    for psi in (three, empty):
        with pytest.raises(tdks.TDKSError):
            ctx.expm(psi, 0.1)


def _atom_initial_state():
    cfg = synth.config1()
    import os
    gs = np.load(os.path.join(os.path.dirname(__file__), "golden", f"gs_{cfg.name}.npz"))
    m = Mesh.from_config(cfg)
    psi0 = kick(m, gs["psibar"].astype(complex), cfg.kick, cfg.kick_dir)
    return cfg, m, psi0


def test_magnus_steps_atom_workload():
    cfg, m, psi0 = _atom_initial_state()
    ctx = _ctx(cfg)
    prop = Propagator.from_config(cfg, m)
    d0 = prop.init(psi0)
    g = _cuda(psi0)
    np.testing.assert_allclose(ctx.init_propagation(g), d0, rtol=1e-12, atol=1e-14)
    ref = psi0
    for n in range(3):
        ref, dref, info = prop.magnus_step(ref, cfg.dt)
        st = ctx.magnus_step(g, cfg.dt, tol=cfg.tol, k_max=cfg.k_max)
        assert st["k_full_max"] == max(max(k) for k in info["k_full"])
        assert _rel(g.cpu().numpy(), ref) < 1e-10
        assert abs(st["dipole"][2] - dref[2]) < 1e-10 * abs(dref[2] - d0[2]) + 1e-13


def test_magnus_steps_atom_workload_df64():
    """Double-float runs: contractions, Krylov recombination and the density
    interpolation in double-float; recurrence, small exponential, Poisson and the
    density and dipole sums in FP64."""
    from paper_1810_13130_gb300 import tdks
    cfg, m, psi0 = _atom_initial_state()
    ctx = _ctx(cfg)
    prop = Propagator.from_config(cfg, m)
    d0 = prop.init(psi0)
    g = _cuda(psi0)
    ctx.init_propagation(g)
    ref = psi0
    for n in range(3):
        ref, dref, info = prop.magnus_step(ref, cfg.dt)
        st = ctx.magnus_step(g, cfg.dt, tol=cfg.tol, k_max=cfg.k_max, prec=tdks.DF64)
        assert _rel(g.cpu().numpy(), ref) < 1e-10
        assert abs(st["dipole"][2] - dref[2]) < 1e-10 * abs(dref[2] - d0[2]) + 1e-13


def test_magnus_step_molecule_workload_properties():
    """One predictor-corrector step of the molecule workload (857,375 DoF, 16 orbitals) in
    the launch configuration the benchmark times, checked by properties that hold at any
    size: the kicked orbitals stay orthonormal (the exponential is unitary up to the Krylov
    tolerance), the reported dipole is that of the new density, and the DF64 step gives
    the FP64 orbitals."""
    from paper_1810_13130_gb300 import tdks
    cfg = synth.config2()
    m = Mesh.from_config(cfg)
    psi0 = synth.smooth_orbitals(tuple(m.Ni), cfg.n_orb, seed=1)
    out = {}
    for prec in (tdks.FP64, tdks.DF64):
        ctx = _ctx(cfg)
        g = _cuda(psi0)
        ctx.kick(g, cfg.kick, cfg.kick_dir)
        ctx.init_propagation(g)
        st = ctx.magnus_step(g, cfg.dt, tol=cfg.tol, k_max=cfg.k_max, prec=prec)
        d = ctx.dipole(ctx.density(g))
        out[prec] = (g.cpu().numpy(), st, d)
        ctx.close()
    psi, st, d = out[tdks.FP64]
    gram = psi.conj() @ psi.T
    assert np.abs(gram - np.eye(cfg.n_orb)).max() < 1e-9
    assert st["k_full_max"] >= st["k_half_max"] > 1 and st["substeps"] == 0
    np.testing.assert_allclose(st["dipole"], d, rtol=1e-12, atol=1e-14)
    assert _rel(out[tdks.DF64][0], psi) < 1e-10
    # the DF64 step's double-float preconditioner (exact to ~1e-14): at this CG tolerance
    # (1e-13) the FP64 CG takes at most one more iteration than with the FP64 one
    assert all(a <= b + 1 for a, b in zip(out[tdks.DF64][1]["cg_iters"], st["cg_iters"]))


def test_magnus_step_with_field_small_system():
    cfg = synth.small_config(3, 2, 2, p=3, n_orb=2)
    m = Mesh.from_config(cfg)
    psi0 = synth.smooth_orbitals(tuple(m.Ni), 2, seed=4)
    ctx = _ctx(cfg)
    prop = Propagator.from_config(cfg, m)
    prop.init(psi0)
    g = _cuda(psi0)
    ctx.init_propagation(g)
    E = lambda t: np.array([0.02 * np.sin(t), 0.0, 0.01])
    ref = psi0
    for n in range(3):
        t0 = n * cfg.dt
        ref, dref, _ = prop.magnus_step(ref, cfg.dt, E(t0 + cfg.dt / 4), E(t0 + cfg.dt / 2))
        st = ctx.magnus_step(g, cfg.dt, E(t0 + cfg.dt / 4), E(t0 + cfg.dt / 2))
        assert _rel(g.cpu().numpy(), ref) < 1e-10
        np.testing.assert_allclose(st["dipole"], dref, rtol=1e-9, atol=1e-12)


def test_propagate_host_equals_device_path():
    cfg = synth.small_config(2, 2, 3, p=3, n_orb=2)
    m = Mesh.from_config(cfg)
    psi0 = synth.smooth_orbitals(tuple(m.Ni), 2, seed=5)
    a = _ctx(cfg)
    g = _cuda(psi0)
    a.init_propagation(g)
    dips = [a.magnus_step(g, cfg.dt)["dipole"] for _ in range(2)]
    b = _ctx(cfg)
    hin = torch.from_numpy(psi0).pin_memory()
    hout = torch.empty_like(hin).pin_memory()
    dh = b.propagate_host(hin, hout, 2, cfg.dt)
    assert torch.equal(hout, g.cpu())
    np.testing.assert_array_equal(dh, np.array(dips))
