"""The allocation-free block inverse (negf_zinv_batched_noalloc) against the ordinary one.

Callers that cannot allocate device memory at call time (their device memory is owned by an
arena reserved at start-up, or they must not call cudaMalloc after initialisation) use the
variant whose scratch is a fixed device array inside the library.  It must give the same
inverses as negf_zinv_batched (FP64 form) on consecutive calls, which share that array.
This file is collected last so that a failure here does not hide the other tests.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
negf = pytest.importorskip("paper_1510_04686_gb300")

pytestmark = pytest.mark.gpu


def _problem(seed, nb, n):
    rng = np.random.default_rng(seed)
    H = (rng.normal(size=(nb, n, n)) + 1j * rng.normal(size=(nb, n, n))) / np.sqrt(2 * n)
    H = 0.5 * (H + np.swapaxes(H, 1, 2).conj())
    z = (0.2 + 1e-3j) + 0.1 * np.arange(nb)
    return z[:, None, None] * np.eye(n) - H


@pytest.mark.parametrize("n", [48, 200])
def test_noalloc_inverse_matches_workspace_inverse(n):
    negf._build.build()
    lib = negf.library()
    nb = 5
    for call, seed in enumerate((11, 12)):  # two calls in a row share the scratch array
        M = _problem(seed + n, nb, n)
        ref, st_ref = negf.zinv(torch.as_tensor(M.copy(), device="cuda"), precision=negf.PREC_FP64)
        Md = torch.as_tensor(M.copy(), device="cuda")
        X = torch.empty_like(Md)
        st = torch.full((nb,), -1, dtype=torch.int32, device="cuda")
        stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        rc = lib.negf_zinv_batched_noalloc(nb, n, ctypes.c_void_p(Md.data_ptr()),
                                           ctypes.c_void_p(X.data_ptr()),
                                           ctypes.c_void_p(st.data_ptr()), stream)
        assert rc == 0, f"call {call}: status {rc}"
        torch.cuda.synchronize()
        X = X.cpu().numpy()
        ref = ref.cpu().numpy()
        assert np.all(st.cpu().numpy() == 0) and np.all(st_ref.cpu().numpy() == 0)
        # same elimination as the workspace form; tolerance of the FP64 block tests
        for p in range(nb):
            assert np.abs(X[p] - ref[p]).max() <= 1e-12 * np.abs(ref[p]).max()
        assert np.allclose(X @ M, np.eye(n), atol=1e-9)


def test_noalloc_small_blocks_need_no_scratch():
    """Blocks of n <= 106 are eliminated in shared memory, so any batch size is accepted: a
    batch whose panel scratch would exceed the fixed array still runs and matches."""
    negf._build.build()
    lib = negf.library()
    n, nb = 48, 2000
    M = _problem(21, nb, n)
    ref, _ = negf.zinv(torch.as_tensor(M.copy(), device="cuda"), precision=negf.PREC_FP64)
    Md = torch.as_tensor(M.copy(), device="cuda")
    X = torch.empty_like(Md)
    st = torch.full((nb,), -1, dtype=torch.int32, device="cuda")
    rc = lib.negf_zinv_batched_noalloc(nb, n, ctypes.c_void_p(Md.data_ptr()),
                                       ctypes.c_void_p(X.data_ptr()),
                                       ctypes.c_void_p(st.data_ptr()),
                                       ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 0
    torch.cuda.synchronize()
    assert np.all(st.cpu().numpy() == 0)
    X, ref = X.cpu().numpy(), ref.cpu().numpy()
    assert np.abs(X - ref).max() <= 1e-12 * np.abs(ref).max()


def test_noalloc_rejects_oversize_batch():
    negf._build.build()
    lib = negf.library()
    n, nb = 1024, 4096  # far beyond the fixed scratch
    fake = ctypes.c_void_p(256)
    rc = lib.negf_zinv_batched_noalloc(nb, n, fake, fake, fake, None)
    assert rc == 3  # NEGF_ERR_NOMEM, before any launch
