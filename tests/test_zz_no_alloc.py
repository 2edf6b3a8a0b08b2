"""tdks_dipole_noalloc, the entry point that allocates no device memory.

It serves callers that cannot allocate (their device memory belongs to another
allocator with a fixed budget, or they must not allocate once running).  The
check: through the C ABI, two calls in a row agree with the context-based
tdks_dipole on the same density, within the 1e-12 relative tolerance the other
FP64 reductions use.  This file sorts last so that a run stopping at the first
failure has already run every other test.
"""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_dipole_noalloc_matches_context_dipole_twice():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1810_13130_gb300.build import build
    build()
    from paper_1810_13130_gb300 import tdks
    results = []
    for cfg in (synth.small_config(3, 2, 4, p=4, n_orb=2, graded=True), synth.config1()):
        ctx = tdks.Context.from_config(cfg)
        n_i = tuple(n * cfg.p - 1 for n in (cfg.nx, cfg.ny, cfg.nz))
        psi = torch.from_numpy(synth.smooth_orbitals(n_i, cfg.n_orb, seed=9)).cuda()
        ctx.kick(psi, 0.3, (1.0, -0.5, 0.25))
        rho = ctx.density(psi)
        ref = ctx.dipole(rho)
        for _ in range(2):
            got = tdks.dipole_noalloc(rho, cfg.X, cfg.Y, cfg.Z, cfg.p)
            scale = max(np.abs(ref).max(), 1e-300)
            assert np.abs(got - ref).max() <= 1e-12 * scale + 1e-15, (got, ref)
            results.append(got)
        ctx.close()
    assert not np.array_equal(results[0], results[2])     # different meshes, different dipoles


def test_dipole_noalloc_rejects_oversize_mesh():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1810_13130_gb300 import tdks
    rho = torch.zeros(8, dtype=torch.float64, device="cuda")
    big = np.linspace(0, 1, 14000)
    with pytest.raises(tdks.TDKSError):
        tdks.dipole_noalloc(rho, big, big, big, 1)
