"""helrm_rescale_noalloc: the rescale for callers that cannot allocate device
memory (their GPU memory belongs to another allocator, or an allocation's
implicit synchronisation is not allowed where they run).  It must give the
same ciphertext as helrm_rescale, bit for bit, on consecutive calls that
share its static scratch array.  This file is collected last so a failure here
cannot hide the other tests; it also passes alone in a fresh process."""
import numpy as np
import pytest

from helpers import gpu_ctx

pytestmark = pytest.mark.gpu


def _random_ct(primes, level, n, seed):
    rng = np.random.default_rng(seed)
    return np.stack([np.stack([rng.integers(0, primes[i], n, dtype=np.uint64) for i in range(level + 1)])
                     for _ in range(2)])


def test_noalloc_rescale_matches_rescale_twice():
    import torch

    from paper_2506_18150_gb300 import helrm as H
    from paper_2506_18150_gb300 import synthetic as syn
    pr = syn.PARAMS["full"]                       # N = 2^16: two polynomials fill the scratch exactly
    ctx = gpu_ctx(pr)
    primes, _ = H.helrm_ctx_primes(ctx)
    n = 1 << pr["log_n"]
    for call, level in enumerate([5, 20]):
        coeffs = _random_ct(primes, level, n, 100 + call)
        # the existing entry point
        ref = H.helrm_rescale(ctx, H.helrm_ct_import(ctx, coeffs, level, 2.0**40))
        want, lvl, _ = H.helrm_ct_export(ctx, ref)
        assert lvl == level - 1
        # the allocation-free one, on caller-owned device buffers in the NTT domain
        d_in = torch.from_numpy(coeffs.reshape(-1).view(np.int64).copy()).cuda()
        for p in range(2):
            H.helrm_ntt(ctx, d_in.data_ptr() + p * (level + 1) * n * 8, level + 1, 0, False)
        d_out = torch.zeros(2 * level * n, dtype=torch.int64, device="cuda")
        H.helrm_rescale_noalloc(ctx, d_in.data_ptr(), d_out.data_ptr(), level, 2)
        for p in range(2):
            H.helrm_ntt(ctx, d_out.data_ptr() + p * level * n * 8, level, 0, True)
        H.helrm_ctx_synchronize(ctx)
        got = d_out.cpu().numpy().view(np.uint64).reshape(2, level, n)
        assert np.array_equal(got, want), f"call {call}: differs from helrm_rescale"


def test_noalloc_rescale_rejects_oversize():
    import torch

    from paper_2506_18150_gb300 import helrm as H
    from paper_2506_18150_gb300 import synthetic as syn
    pr = syn.PARAMS["full"]
    ctx = gpu_ctx(pr)
    n = 1 << pr["log_n"]
    buf = torch.zeros(3 * 3 * n, dtype=torch.int64, device="cuda")
    with pytest.raises(H.HelrmError) as e:
        H.helrm_rescale_noalloc(ctx, buf.data_ptr(), buf.data_ptr(), 2, 3)   # 3 x 2^16 words > scratch
    assert e.value.name == "HELRM_E_INVAL"
