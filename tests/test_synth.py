"""The seeded synthetic inputs: deterministic, in the documented ranges, and with the
properties the tests and the benchmark rely on (no method arithmetic here)."""
import numpy as np

import synth


def test_smooth_orbitals_are_orthonormal_and_seeded():
    a = synth.smooth_orbitals((9, 7, 8), 5, seed=3)
    b = synth.smooth_orbitals((9, 7, 8), 5, seed=3)
    c = synth.smooth_orbitals((9, 7, 8), 5, seed=4)
    assert a.shape == (5, 9 * 7 * 8) and a.dtype == np.complex128
    np.testing.assert_array_equal(a, b)
    assert np.abs(a - c).max() > 1e-3
    np.testing.assert_allclose(a.conj() @ a.T, np.eye(5), atol=1e-13)


def test_random_psi_unit_norm_and_seeded():
    a = synth.random_psi(3, 100, seed=9)
    np.testing.assert_allclose(np.linalg.norm(a, axis=1), 1.0, rtol=1e-14)
    np.testing.assert_array_equal(a, synth.random_psi(3, 100, seed=9))


def test_batch_workload_in_its_ranges():
    cfgs, dts, dirs = synth.config5()
    assert len(cfgs) == 64
    for c, dt, d in zip(cfgs, dts, dirs):
        n = len(c.X) - 1
        assert 4 <= n <= 12 and 4 <= c.p <= 8 and 1 <= c.n_orb <= 8
        assert 1 <= len(c.atom_Z) <= 4 and set(c.atom_Z) <= {1.0, 2.0, 3.0, 4.0}
        assert np.all(np.abs(c.atom_R) <= n / 3 + 1e-12)
        assert dt in (0.02, 0.05, 0.1) and c.dt == dt
        assert abs(np.linalg.norm(d) - 1.0) < 1e-14
        np.testing.assert_allclose(np.diff(c.X), 2.0)          # 2-bohr elements
    again, _, _ = synth.config5()
    assert [c.name for c in again] == [c.name for c in cfgs]


def test_graded_mesh_of_the_all_electron_workload():
    c = synth.config3()
    for b in (c.X, c.Y, c.Z):
        assert len(b) == 25 and b[0] == -20.0 and b[-1] == 20.0
        h = np.diff(b)
        np.testing.assert_allclose(h, h[::-1], rtol=1e-13)       # symmetric about 0
        np.testing.assert_allclose(h[12:][1:] / h[12:][:-1], 1.25, rtol=1e-12)   # growth 1.25 outward
    assert c.p == 8 and c.n_orb == 5 and list(c.atom_Z) == [6.0, 1.0, 1.0, 1.0, 1.0]
    np.testing.assert_allclose(np.linalg.norm(c.atom_R[1:], axis=1), 2.05, rtol=1e-14)


def test_molecule_workload_atoms():
    c = synth.config2()
    assert (c.p, c.n_orb, len(c.X) - 1) == (6, 16, 16) and len(c.atom_Z) == 8
    r = np.linalg.norm(c.atom_R, axis=1)
    assert r.max() <= 6.0
    dmin = min(np.linalg.norm(c.atom_R[i] - c.atom_R[j])
               for i in range(8) for j in range(i + 1, 8))
    assert dmin >= 1.5
