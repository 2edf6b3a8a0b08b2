"""Write the FP64 oracle dipole series that the GPU paths are checked against.

Calls only the CPU oracle.  Two workloads, each started from an oracle ground
state, kicked by exp(-i kappa r.d) (Sec. VII.A) and propagated by the
predictor-corrector Magnus step (Eqs. 25-26, Sec. VI.B) with adaptive Lanczos
(Eqs. 36-38):

* atom: the 2-electron soft-Coulomb atom (6^3 elements, p = 4, 1 orbital), its
  full 100 steps of dt 0.05 from tests/golden/gs_atom_soft_Z2_6x6x6_p4.npz;
* mid: the 8-orbital erf-pseudopotential molecule of synth.config_mid()
  (8^3 elements, p = 6, 103,823 DoF, 4 atoms), 50 steps of dt 0.1, from a
  ground state of 20 SCF iterations written here first
  (tests/golden/gs_molecule_erf4_8x8x8_p6.npz).

Per workload it stores the dipoles d(t_n), n = 0..N (Sec. V, Eq. 30), the
Krylov dimension of both exponentials of every step and orbital, the Poisson
CG iteration counts, the final orbitals, and the oracle's wall time on one
thread of the machine that ran it.  To keep the files small, a ground state
written here is stored rounded to float32 (the propagation starts from exactly
that rounded state), and for more than 2e5 orbital values the final orbitals
are kept as a seeded sample of 8192 entries per orbital plus their projections
<R_k, psi_a> onto three seeded random unit vectors R_k (synth.random_psi).

    OMP_NUM_THREADS=1 python tests/golden/make_dipole_series.py atom|mid
"""
import os
import platform
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import synth  # noqa: E402
from oracle.ground_state import scf  # noqa: E402
from oracle.mesh import Mesh  # noqa: E402
from oracle.propagate import Propagator, kick, nuclear_potential  # noqa: E402

CG_TOL = 1e-13


def ground_state(cfg, mesh, n_iter):
    path = os.path.join(HERE, f"gs_{cfg.name}.npz")
    if os.path.exists(path):
        return np.load(path)["psibar"].astype(complex)
    vn = nuclear_potential(mesh, cfg.nuc_kind, cfg.atom_R, cfg.atom_Z, cfg.nuc_param)
    psi, vals, _ = scf(mesh, vn, cfg.occ, cfg.n_orb, n_iter=n_iter, mix=0.5)
    for a in range(psi.shape[0]):          # sign: largest component positive
        if psi[a, np.argmax(np.abs(psi[a]))] < 0:
            psi[a] = -psi[a]
    psi = psi.astype(np.float32)
    np.savez_compressed(path, psibar=psi, eigenvalues=vals, scf_iterations=n_iter)
    print(path, vals, flush=True)
    return psi.astype(complex)


def final_orbitals(cfg, psi):
    """The final orbitals in full, or (large systems) a seeded sample and projections."""
    if psi.size <= 200000:
        return {"psibar_final": psi}
    rng = np.random.default_rng(cfg.seed + 1)
    idx = np.sort(rng.choice(psi.shape[1], 8192, replace=False))
    R = synth.random_psi(3, psi.shape[1], seed=cfg.seed + 2)
    return {"final_sample_idx": idx, "final_sample": psi[:, idx], "final_proj": psi @ R.conj().T,
            "final_proj_seed": cfg.seed + 2}


def series(cfg, n_scf):
    mesh = Mesh.from_config(cfg)
    psi = ground_state(cfg, mesh, n_scf)
    prop = Propagator.from_config(cfg, mesh, cg_tol=CG_TOL)
    psi = kick(mesh, psi, cfg.kick, cfg.kick_dir)
    t0 = time.perf_counter()
    dip = [prop.init(psi)]
    kh, kf = [], []
    for n in range(cfg.n_steps):
        psi, d, info = prop.magnus_step(psi, cfg.dt)
        dip.append(d)
        kh.append([sum(k) for k in info["k_half"]])
        kf.append([sum(k) for k in info["k_full"]])
        if n % 10 == 0:
            print(f"{cfg.name} step {n} k {kh[-1]} {kf[-1]} {time.perf_counter() - t0:.1f}s",
                  flush=True)
    wall = time.perf_counter() - t0
    out = os.path.join(HERE, f"series_{cfg.name}.npz")
    np.savez_compressed(out, dipole=np.array(dip), k_half=np.array(kh, dtype=np.int32),
                        k_full=np.array(kf, dtype=np.int32),
                        cg_iters=np.array(prop.cg_iters, dtype=np.int32), **final_orbitals(cfg, psi),
                        n_steps=cfg.n_steps, dt=cfg.dt, tol=cfg.tol, k_max=cfg.k_max,
                        kappa=cfg.kick, kick_dir=np.array(cfg.kick_dir), cg_tol=CG_TOL,
                        oracle_wall_s=wall, oracle_threads=1,
                        oracle_host=f"{platform.machine()} {platform.processor() or ''}".strip())
    print(out, f"{wall:.1f}s", flush=True)


def main():
    which = sys.argv[1] if len(sys.argv) > 1 else "atom"
    if which == "atom":
        series(synth.config1(), 50)
    elif which == "mid":
        series(synth.config_mid(), 20)
    else:
        raise SystemExit("usage: make_dipole_series.py atom|mid")


if __name__ == "__main__":
    main()
