"""helrm_rescale_noalloc: the rescale for callers that cannot allocate device
memory (their GPU memory belongs to another allocator, or an allocation's
implicit synchronisation is not allowed where they run).  It must give the
same ciphertext as helrm_rescale, bit for bit, on consecutive calls that
share its static scratch array, and the oracle's rescale (round(x / q_l) by
the centred remainder).  This file is collected last so a failure here
cannot hide the other tests; it also passes alone in a fresh process."""
import numpy as np
import pytest

from helpers import gpu_ctx, oracle_params

pytestmark = pytest.mark.gpu


def _random_polys(primes, level, n, n_polys, seed):
    rng = np.random.default_rng(seed)
    return np.stack([np.stack([rng.integers(0, primes[i], n, dtype=np.uint64) for i in range(level + 1)])
                     for _ in range(n_polys)])


def _noalloc(ctx, coeffs, level, n):
    """coeffs [n_polys][level+1][n] (coefficient domain) -> the call's output,
    back in the coefficient domain, [n_polys][level][n]."""
    import torch

    from paper_2506_18150_gb300 import helrm as H
    n_polys = coeffs.shape[0]
    d_in = torch.from_numpy(coeffs.reshape(-1).view(np.int64).copy()).cuda()
    for p in range(n_polys):
        H.helrm_ntt(ctx, d_in.data_ptr() + p * (level + 1) * n * 8, level + 1, 0, False)
    d_out = torch.zeros(n_polys * level * n, dtype=torch.int64, device="cuda")
    H.helrm_rescale_noalloc(ctx, d_in.data_ptr(), d_out.data_ptr(), level, n_polys)
    for p in range(n_polys):
        H.helrm_ntt(ctx, d_out.data_ptr() + p * level * n * 8, level, 0, True)
    H.helrm_ctx_synchronize(ctx)
    return d_out.cpu().numpy().view(np.uint64).reshape(n_polys, level, n)


def test_noalloc_rescale_matches_rescale_twice():
    from paper_2506_18150_gb300 import helrm as H
    from paper_2506_18150_gb300 import synthetic as syn
    pr = syn.PARAMS["full"]                       # N = 2^16: two polynomials fill the scratch exactly
    ctx = gpu_ctx(pr)
    primes, _ = H.helrm_ctx_primes(ctx)
    n = 1 << pr["log_n"]
    for call, level in enumerate([5, 20]):
        coeffs = _random_polys(primes, level, n, 2, 100 + call)
        # the existing entry point
        ref = H.helrm_rescale(ctx, H.helrm_ct_import(ctx, coeffs, level, 2.0**40))
        want, lvl, _ = H.helrm_ct_export(ctx, ref)
        assert lvl == level - 1
        got = _noalloc(ctx, coeffs, level, n)
        assert np.array_equal(got, want), f"call {call}: differs from helrm_rescale"


@pytest.mark.parametrize("level,n_polys", [(1, 1), (1, 2), (3, 1), (5, 2)])
def test_noalloc_rescale_matches_oracle(level, n_polys):
    from oracle import ckks
    from paper_2506_18150_gb300 import synthetic as syn
    pr = syn.reduced_params(12, 5)
    p = oracle_params(pr)
    ctx = gpu_ctx(pr)
    n = p.N
    for call in range(2):                          # two calls in a row on the shared scratch
        coeffs = _random_polys(p.q, level, n, n_polys, 300 + 10 * level + call)
        got = _noalloc(ctx, coeffs, level, n)
        for k in range(n_polys):
            want = ckks.rescale_poly(p, coeffs[k], level)
            assert np.array_equal(got[k], want), f"level {level}, poly {k}, call {call}: differs from the oracle"


def test_noalloc_rescale_allocates_nothing():
    """On a fresh context the device's free memory is the same before and after
    the first call: the scratch array and the kernels were loaded when the
    context was created."""
    import torch

    from paper_2506_18150_gb300 import helrm as H
    from paper_2506_18150_gb300 import synthetic as syn
    pr = syn.PARAMS["full"]
    ctx = gpu_ctx(pr)
    n = 1 << pr["log_n"]
    level = 4
    d_in = torch.zeros(2 * (level + 1) * n, dtype=torch.int64, device="cuda")
    d_out = torch.zeros(2 * level * n, dtype=torch.int64, device="cuda")
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    H.helrm_rescale_noalloc(ctx, d_in.data_ptr(), d_out.data_ptr(), level, 2)
    H.helrm_ctx_synchronize(ctx)
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, f"device free memory changed by {free0 - free1} bytes"


def test_noalloc_rescale_rejects_oversize_and_overlap():
    import torch

    from paper_2506_18150_gb300 import helrm as H
    from paper_2506_18150_gb300 import synthetic as syn
    pr = syn.PARAMS["full"]
    ctx = gpu_ctx(pr)
    n = 1 << pr["log_n"]
    buf = torch.zeros(3 * 3 * n, dtype=torch.int64, device="cuda")
    with pytest.raises(H.HelrmError) as e:
        H.helrm_rescale_noalloc(ctx, buf.data_ptr(), buf.data_ptr() + 6 * n * 8, 2, 3)   # 3 x 2^16 words > scratch
    assert e.value.name == "HELRM_E_INVAL"
    # in: 2 x 3 limbs from word 0; out: 2 x 2 limbs starting inside the input
    with pytest.raises(H.HelrmError) as e:
        H.helrm_rescale_noalloc(ctx, buf.data_ptr(), buf.data_ptr() + 5 * n * 8, 2, 2)
    assert e.value.name == "HELRM_E_INVAL"
    # adjacent, not overlapping: accepted
    H.helrm_rescale_noalloc(ctx, buf.data_ptr(), buf.data_ptr() + 6 * n * 8, 2, 1)
    H.helrm_ctx_synchronize(ctx)
