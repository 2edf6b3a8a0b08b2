"""Host-side logic of bench.py (no GPU): the dipole-error definition and the rule that
the roofline's DRAM traffic is taken from a committed ncu summary only while the
element-kernel source it was captured from is unchanged."""
import hashlib
import os

import numpy as np

import bench


def test_dipole_error_is_relative_to_the_induced_dipole():
    # ref: d(t) = d0 + a(t); d = ref + e(t): error = max|e| / max|a|  (Sec. V, Eq. 30)
    t = np.linspace(0.0, 1.0, 11)
    ref = np.stack([0.5 + 1e-3 * np.sin(3 * t), -0.2 + 2e-3 * t, 0.1 + 0 * t], axis=1)
    e = np.zeros_like(ref)
    e[4, 1] = 3e-9
    np.testing.assert_allclose(bench.dipole_err(ref + e, ref), 3e-9 / np.abs(ref - ref[0]).max(), rtol=1e-6)
    assert bench.dipole_err(ref, ref) == 0.0


def test_profile_traffic_follows_the_kernel_source(tmp_path, monkeypatch):
    src = open(os.path.join(bench.ROOT, "paper_1810_13130_gb300", "csrc", "elements.cu"), "rb").read()
    sha = hashlib.sha256(src).hexdigest()[:16]
    good = tmp_path / "good.txt"
    good.write_text(f"# summary\nelements_cu_sha256_16: {sha}\ndram_bytes_per_launch_full_size: 123.5e6\n")
    stale = tmp_path / "stale.txt"
    stale.write_text("elements_cu_sha256_16: 0000000000000000\ndram_bytes_per_launch_full_size: 9e6\n")
    monkeypatch.setattr(bench, "PROFILES", {"fp64": str(good), "df64": str(stale)})
    assert bench.profile_traffic("fp64") == 123.5e6
    assert bench.profile_traffic("df64") is None          # captured from another source
    assert bench.profile_traffic("fp32") is None          # no summary
