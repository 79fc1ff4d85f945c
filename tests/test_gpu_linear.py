"""GPU parity of the double-hoisted BSGS matvec and the packed embedding
lookup: bit-exact against the oracle when both use the oracle's integer
diagonals, within 1e-3 of the cleartext product with the library's own
encoder; the tiny workload (1024 x 16 table in base 32) packed and unpacked."""
import numpy as np
import pytest

from helpers import assert_ct_equal, gpu_ctx, oracle_params

pytestmark = pytest.mark.gpu

SHAPES = [(16, 64), (64, 16), (32, 32), (1, 32), (10, 3), (5, 7), (48, 200)]


@pytest.fixture(scope="module")
def env():
    from paper_2506_18150_gb300 import synthetic as syn
    pr = syn.reduced_params(12, 4)
    return gpu_ctx(pr), oracle_params(pr)


def _keys(ctx, p, steps, seed):
    from oracle import ckks
    from paper_2506_18150_gb300 import helrm as H
    sk, evk = H.helrm_keygen(ctx, seed, steps)
    sk_o, keys_o = ckks.keygen(p, seed, rot_steps=steps, relin=False)
    return sk, evk, sk_o, keys_o


@pytest.mark.parametrize("shape", SHAPES)
def test_matvec_bit_exact_and_accurate(env, shape):
    from oracle import ckks, dlrm, linear
    from paper_2506_18150_gb300 import helrm as H
    ctx, p = env
    rows, cols = shape
    rng = np.random.default_rng(rows * 1000 + cols)
    W = rng.normal(0, 0.3, shape)
    W[:, rng.integers(0, cols)] = 0.0                       # a zero column (ragged content)
    x = rng.uniform(-1, 1, cols)
    ip, op = linear.pow2ceil(cols), linear.pow2ceil(rows)
    lvl = 3
    pm_o = linear.prepare(p, W, ip, op, lvl, p.delta, p.delta)
    pm = H.helrm_ptmat_prepare(ctx, W, ip, op, lvl, p.delta, p.delta)
    info = H.helrm_ptmat_info(ctx, pm)
    assert (info["D"], info["n1"], info["n2"]) == (pm_o.layout.D, pm_o.layout.n1, pm_o.layout.n2)
    assert info["nonzero"] == len(pm_o.pts) and info["folds"] == len(pm_o.layout.folds)
    steps = linear.rotation_steps(pm_o)
    assert H.helrm_ptmat_rotations(ctx, pm) == steps
    sk, evk, sk_o, keys_o = _keys(ctx, p, steps, 5)
    m = ckks.encode_real(p, dlrm.replicate(x, ip, p.n), p.delta)
    ct = H.helrm_encrypt(ctx, evk, H.helrm_pt_import(ctx, m, lvl, p.delta), 9)
    ct_o = ckks.encrypt(p, keys_o, m, lvl, p.delta, 9)
    want = linear.matvec_cleartext(W, x, ip, op, p.n)
    # (1) the library's own encoding: accurate
    out = H.helrm_ptct_matvec(ctx, evk, pm, ct)
    assert H.helrm_ct_info(ctx, out)[0] == lvl - 1
    assert np.max(np.abs(H.helrm_decrypt(ctx, sk, out, p.n) - want)) < 1e-3
    # (2) the oracle's integer diagonals: bit-exact
    H.helrm_ptmat_import(ctx, pm, np.stack([pm_o.pts[k] for k in pm_o.ordered_keys()]).astype(np.int64))
    out2 = H.helrm_ptct_matvec(ctx, evk, pm, ct)
    assert_ct_equal(ctx, out2, linear.matvec(p, keys_o, pm_o, ct_o))


def test_matvec_missing_key_and_level(env):
    from oracle import linear
    from paper_2506_18150_gb300 import helrm as H
    ctx, p = env
    W = np.random.default_rng(1).normal(0, 0.3, (16, 16))
    pm = H.helrm_ptmat_prepare(ctx, W, 16, 16, 2, p.delta, p.delta)
    sk, evk = H.helrm_keygen(ctx, 3, [1, 2])                   # not enough keys
    ct = H.helrm_encrypt(ctx, evk, H.helrm_encode(ctx, np.zeros(16), 2, p.delta), 1)
    with pytest.raises(H.HelrmError) as e:
        H.helrm_ptct_matvec(ctx, evk, pm, ct)
    assert e.value.name == "HELRM_E_NOKEY"
    ct3 = H.helrm_encrypt(ctx, evk, H.helrm_encode(ctx, np.zeros(16), 3, p.delta), 1)
    with pytest.raises(H.HelrmError) as e:
        H.helrm_ptct_matvec(ctx, evk, pm, ct3)
    assert e.value.name == "HELRM_E_LEVEL"


@pytest.fixture(scope="module")
def tiny():
    from oracle import ckks, dlrm, linear
    from paper_2506_18150_gb300 import helrm as H
    from paper_2506_18150_gb300 import synthetic as syn
    pr = syn.PARAMS["tiny"]
    ctx, p = gpu_ctx(pr), oracle_params(pr)
    C = syn.tiny_table(0)
    M = dlrm.lookup_matrix(C, 32, 1024)
    pm_o = linear.prepare(p, M, 64, 16, 1, p.delta, p.delta)
    pm_d = [linear.prepare(p, M[:, 32 * j: 32 * j + 32], 32, 16, 1, p.delta, p.delta) for j in range(2)]
    steps = sorted(set(linear.rotation_steps(pm_o)) | set(linear.rotation_steps(pm_d[0])))
    sk, evk = H.helrm_keygen(ctx, 0, steps)
    sk_o, keys_o = ckks.keygen(p, 0, rot_steps=steps, relin=False)
    emb = H.helrm_emb_prepare(ctx, [1024], 32, 0, 16, [C], 0, 16, 1, p.delta, p.delta)
    return ctx, p, C, M, pm_o, pm_d, sk, evk, sk_o, keys_o, emb


def test_tiny_lookup_all_paths(tiny):
    """Both selectors in one ciphertext (the paper's packing) and each selector
    its own ciphertext; sampled indices incl. 0 and 1023; bit-exact vs oracle
    with imported diagonals; within 1e-3 of the gather with the GPU encoder."""
    from oracle import ckks, dlrm, linear
    from paper_2506_18150_gb300 import helrm as H
    ctx, p, C, M, pm_o, pm_d, sk, evk, sk_o, keys_o, emb = tiny
    assert H.helrm_emb_info(ctx, emb) == (64, 64)
    rng = np.random.default_rng(2)
    for i in [0, 1023] + [int(v) for v in rng.integers(0, 1024, 6)]:
        want = C[0][i % 32].astype(np.float64) + C[1][i // 32].astype(np.float64)
        sel = dlrm.replicate(dlrm.selector_vector([1024], 32, [i]), 64, p.n)
        assert np.array_equal(H.helrm_query_pack(ctx, emb, [i], p.n), sel)
        ct = H.helrm_encrypt(ctx, evk, H.helrm_encode(ctx, sel, 1, p.delta), 100 + i)
        out = H.helrm_embedding_lookup(ctx, evk, emb, ct)
        got = H.helrm_decrypt(ctx, sk, out, p.n)
        assert np.max(np.abs(got - np.tile(want, p.n // 16))) < 1e-3
        # separate selectors: sum of two matvecs
        parts = []
        for j in range(2):
            s = dlrm.replicate(sel[32 * j: 32 * j + 32], 32, p.n)
            pm = H.helrm_ptmat_prepare(ctx, M[:, 32 * j: 32 * j + 32], 32, 16, 1, p.delta, p.delta)
            c = H.helrm_encrypt(ctx, evk, H.helrm_encode(ctx, s, 1, p.delta), 7 * i + j)
            parts.append(H.helrm_ptct_matvec(ctx, evk, pm, c))
        got2 = H.helrm_decrypt(ctx, sk, H.helrm_add(ctx, parts[0], parts[1]), 16)
        assert np.max(np.abs(got2 - want)) < 1e-3
    # bit-exact with the oracle's encoding of selector and diagonals
    i = 513
    sel = dlrm.replicate(dlrm.selector_vector([1024], 32, [i]), 64, p.n)
    m = ckks.encode_real(p, sel, p.delta)
    ct = H.helrm_encrypt(ctx, evk, H.helrm_pt_import(ctx, m, 1, p.delta), 5)
    pm = H.helrm_ptmat_prepare(ctx, M, 64, 16, 1, p.delta, p.delta)
    H.helrm_ptmat_import(ctx, pm, np.stack([pm_o.pts[k] for k in pm_o.ordered_keys()]).astype(np.int64))
    ct_o = ckks.encrypt(p, keys_o, m, 1, p.delta, 5)
    assert_ct_equal(ctx, H.helrm_ptct_matvec(ctx, evk, pm, ct), linear.matvec(p, keys_o, pm_o, ct_o))


def test_uncompressed_1024_row_lookup(tiny):
    """The plain one-hot lookup of the same table (1024 selector slots)."""
    from oracle import dlrm
    from paper_2506_18150_gb300 import helrm as H
    ctx, p, C = tiny[0], tiny[1], tiny[2]
    E = np.stack([C[0][i % 32].astype(np.float64) + C[1][i // 32].astype(np.float64) for i in range(1024)])
    emb = H.helrm_emb_prepare(ctx, [1024], 1024, 0, 16, [[E.astype(np.float32)]], 0, 16, 1, p.delta, p.delta)
    assert H.helrm_emb_info(ctx, emb) == (1024, 1024)
    sk, evk = H.helrm_keygen(ctx, 4, [])
    pm = H.helrm_ptmat_prepare(ctx, E.T, 1024, 16, 1, p.delta, p.delta)     # same layout as the lookup
    H.helrm_evk_add_rotations(ctx, sk, evk, H.helrm_ptmat_rotations(ctx, pm))
    for i in [0, 5, 1023]:
        sel = dlrm.replicate(np.eye(1024)[i], 1024, p.n)
        assert np.array_equal(H.helrm_query_pack(ctx, emb, [i], p.n), sel)
        ct = H.helrm_encrypt(ctx, evk, H.helrm_encode(ctx, sel, 1, p.delta), i)
        got = H.helrm_decrypt(ctx, sk, H.helrm_embedding_lookup(ctx, evk, emb, ct), 16)
        assert np.max(np.abs(got - E[i])) < 1e-3
