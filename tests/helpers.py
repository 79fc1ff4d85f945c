"""Shared helpers for the GPU parity tests: build matching library/oracle
contexts, move data between them, and make the oracle's keys in a process
pool.  Nothing here computes the method: the key helper only calls the
oracle's own key functions."""
import multiprocessing as mp
import os
from concurrent.futures import ProcessPoolExecutor

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


def _worker_init(threads):
    os.environ["OMP_NUM_THREADS"] = str(threads)   # before the oracle's OpenMP library loads here


def _switch_key_task(job):
    """One oracle switching key, composed as the oracle's keygen composes it:
    key id 0 = relinearisation (s' = s^2), else the Galois element k (s' = s(X^k))."""
    from oracle import ckks, ring
    pr, seed, k, h = job
    p = oracle_params(pr)
    sk = ckks.secret_key(p, seed, h)
    mods = p.qp_mods(p.L)
    if k == 0:
        s_mod = ring.from_signed(sk.s, mods)
        target = ckks.polymul(p, s_mod, s_mod, mods)
    else:
        target = ring.from_signed(ckks.automorphism_signed(p, sk.s, k), mods)
    return k, ckks.switch_key(p, seed, sk, target, k)


def oracle_keys_pool(pr, seed, steps, h=0, conj=False):
    """The oracle's keys (public, relinearisation, one per rotation step and,
    with conj, the conjugation key; a sparse secret of weight h if h > 0),
    each switching key made by the oracle's own key functions in a
    spawn-started process pool, one key per task; equal to ckks.keygen's."""
    from oracle import ckks
    p = oracle_params(pr)
    sk = ckks.secret_key(p, seed, h)
    keys = ckks.Keys(seed, *ckks.public_key(p, seed, sk))
    gal = sorted({p.galois(st) for st in {int(r) % p.n for r in steps} - {0}})
    if conj:
        gal.append(p.conj_galois())
    jobs = [(pr, seed, 0, h)] + [(pr, seed, k, h) for k in gal]
    cpus = os.cpu_count() or 1
    workers = max(1, min(16, cpus, len(jobs)))
    with ProcessPoolExecutor(workers, mp_context=mp.get_context("spawn"),            # a lost worker raises
                             initializer=_worker_init, initargs=(max(1, cpus // workers),)) as pool:
        for k, sw in pool.map(_switch_key_task, jobs):
            if k == 0:
                keys.relin = sw
            else:
                keys.rot[k] = sw
    return sk, keys
