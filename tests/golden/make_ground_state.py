"""Write the ground-state orbitals of the 2-electron soft-Coulomb atom workload.

Calls only the CPU oracle: 50 SCF iterations (Hartree + LDA) on the 6^3-element,
p = 4 mesh over [-10, 10]^3 with V_N = -2 / sqrt(r^2 + 0.5).  The result is the
initial state psibar^0 (Loewdin basis, before the kick) of the propagation tests.

    python tests/golden/make_ground_state.py
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import synth  # noqa: E402
from oracle.ground_state import scf  # noqa: E402
from oracle.mesh import Mesh  # noqa: E402
from oracle.propagate import nuclear_potential  # noqa: E402


def main():
    cfg = synth.config1()
    mesh = Mesh.from_config(cfg)
    vn = nuclear_potential(mesh, cfg.nuc_kind, cfg.atom_R, cfg.atom_Z, cfg.nuc_param)
    psi, vals, _ = scf(mesh, vn, cfg.occ, cfg.n_orb, n_iter=50, mix=0.5)
    # fix the sign so that the largest component is positive
    for a in range(psi.shape[0]):
        if psi[a, np.argmax(np.abs(psi[a]))] < 0:
            psi[a] = -psi[a]
    out = os.path.join(HERE, f"gs_{cfg.name}.npz")
    np.savez_compressed(out, psibar=psi, eigenvalues=vals)
    print(out, vals)


if __name__ == "__main__":
    main()
