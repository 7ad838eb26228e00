"""The allocation-free Gram-Schmidt entry point (mor_orthonormalize_noalloc)
against the handle-based one (mor_orthonormalize), through the C ABI.

It serves callers that cannot let the library allocate device memory; its
scratch is a fixed array inside the library, shared by all calls.  Two calls
in a row on different inputs must both match the handle-based result (same
kernels, different block counts, so sums are reordered: 1e-12 relative).
This file is collected last so that a run that stops at the first failure
has already run every other test."""
import numpy as np
import pytest

import paper_2003_12759_gb300 as mor

pytestmark = pytest.mark.gpu


def test_noalloc_orthonormalize_matches_handle_version_twice():
    import scipy.sparse as sp
    import torch
    mor.load_library()
    h = mor.mor_create(0)
    try:
        n = 50_001                    # ragged: not a multiple of the 32-row tiles
        # the handle-based entry point needs a system of n rows; its matrix is irrelevant here
        mor.mor_set_system(h, sp.csr_matrix(sp.diags(-np.ones(n))), np.ones((n, 1)), np.ones((n, 1)))
        rng = np.random.default_rng(11)
        for call, k in enumerate((10, 7)):
            X = rng.standard_normal((n, k))
            X[:, 3] += 0.5 * X[:, 2]
            ref = mor.mor_orthonormalize(h, X)
            Xd = torch.from_numpy(np.ascontiguousarray(X.T)).to("cuda").t()   # column-major, stride (1, n)
            assert Xd.stride() == (1, n)
            code = mor.mor_orthonormalize_noalloc(Xd, torch.cuda.current_stream())
            torch.cuda.synchronize()
            assert code == mor.MOR_OK, (call, code)
            got = Xd.cpu().numpy()
            np.testing.assert_allclose(got, ref, rtol=0, atol=1e-12)
            assert np.linalg.norm(got.T @ got - np.eye(k)) <= 1e-13
    finally:
        mor.mor_destroy(h)


def test_noalloc_full_width_and_single_column():
    """k = 64 fills every region of the fixed scratch (all eight column-group
    counters of the Gram kernel, 64 coefficients and norms); k = 1 is the
    one-column case (a contiguous (n, 1) tensor)."""
    import scipy.sparse as sp
    import torch
    mor.load_library()
    h = mor.mor_create(0)
    try:
        n = 4097
        mor.mor_set_system(h, sp.csr_matrix(sp.diags(-np.ones(n))), np.ones((n, 1)), np.ones((n, 1)))
        rng = np.random.default_rng(12)
        for k in (64, 1):
            X = rng.standard_normal((n, k))
            ref = mor.mor_orthonormalize(h, X)
            Xd = torch.from_numpy(np.ascontiguousarray(X.T)).to("cuda").t()
            assert mor.mor_orthonormalize_noalloc(Xd, torch.cuda.current_stream()) == mor.MOR_OK
            torch.cuda.synchronize()
            got = Xd.cpu().numpy()
            np.testing.assert_allclose(got, ref, rtol=0, atol=1e-12)
            assert np.linalg.norm(got.T @ got - np.eye(k)) <= 1e-13
    finally:
        mor.mor_destroy(h)


def test_noalloc_rejects_tensors_it_cannot_read():
    """The binding refuses a tensor whose dtype or layout the C side would
    misread (FP32 data read as FP64 would run past the allocation)."""
    import torch
    mor.load_library()
    with pytest.raises(ValueError):
        mor.mor_orthonormalize_noalloc(torch.zeros((100, 3), dtype=torch.float32, device="cuda").t().contiguous().t())
    with pytest.raises(ValueError):
        mor.mor_orthonormalize_noalloc(torch.zeros((100, 3), dtype=torch.float64, device="cuda"))   # row-major


def test_noalloc_rejects_sizes_beyond_the_limit():
    import torch
    mor.load_library()
    X = torch.zeros((100, 65), dtype=torch.float64, device="cuda").t().contiguous().t()
    assert mor.mor_orthonormalize_noalloc(X) == mor.MOR_EINVAL
