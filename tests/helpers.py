"""Shared helpers for the GPU parity tests: build matching library/oracle
contexts and move data between them.  Nothing here computes the method."""
import numpy as np


def oracle_params(pr):
    from oracle import ckks
    return ckks.Params(pr["log_n"], pr["q_bits"], pr["n_p"], pr["p_bits"], pr["alpha"], pr["log2_scale"])


def gpu_ctx(pr):
    import torch

    from paper_2506_18150_gb300 import helrm as H
    return H.helrm_ctx_create(pr["log_n"], pr["q_bits"], pr["n_p"], pr["p_bits"], pr["alpha"],
                              pr["log2_scale"], device=0, stream=torch.cuda.current_stream().cuda_stream)


def bitrev_perm(log_n):
    n = 1 << log_n
    return np.array([int(f"{i:0{log_n}b}"[::-1], 2) for i in range(n)], dtype=np.int64)


def export_ct(ctx, ct):
    from paper_2506_18150_gb300 import helrm as H
    coeffs, lvl, scale = H.helrm_ct_export(ctx, ct)
    return coeffs, lvl, scale


def assert_ct_equal(ctx, ct_gpu, ct_or):
    coeffs, lvl, scale = export_ct(ctx, ct_gpu)
    assert lvl == ct_or.level, (lvl, ct_or.level)
    assert np.array_equal(coeffs[0], ct_or.c0), "c0 differs"
    assert np.array_equal(coeffs[1], ct_or.c1), "c1 differs"
    assert abs(scale - ct_or.scale) <= 1e-12 * abs(ct_or.scale), (scale, ct_or.scale)


def import_ct(ctx, ct_or):
    from paper_2506_18150_gb300 import helrm as H
    return H.helrm_ct_import(ctx, np.stack([ct_or.c0, ct_or.c1]), ct_or.level, ct_or.scale)


def as_signed(m):
    return np.array([int(x) for x in m], dtype=np.int64)
