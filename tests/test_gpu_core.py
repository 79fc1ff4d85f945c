"""GPU parity of the CKKS layer against the oracle, through the C-ABI:
primes, NTT, encryption, decryption, rescale, rotation (single and hoisted),
ct x ct multiplication, and the error paths.  Ciphertexts are compared
bit-exactly in the coefficient domain; the encoder within one unit."""
import numpy as np
import pytest

from helpers import assert_ct_equal, bitrev_perm, gpu_ctx, import_ct, oracle_params

pytestmark = pytest.mark.gpu

STEPS = [1, 3, -1, 100, -7, 5]


@pytest.fixture(scope="module")
def env():
    from oracle import ckks
    from paper_2506_18150_gb300 import helrm as H
    from paper_2506_18150_gb300 import synthetic as syn
    pr = syn.reduced_params(12, 4)          # N = 2^12, q_0 60-bit + 4 x 40-bit, K = 3, alpha = 3
    ctx = gpu_ctx(pr)
    p = oracle_params(pr)
    sk, evk = H.helrm_keygen(ctx, 99, STEPS)
    sk_o, keys_o = ckks.keygen(p, 99, rot_steps=STEPS)
    return ctx, p, sk, evk, sk_o, keys_o


def fresh(env, level, seed, z=None):
    from oracle import ckks
    from paper_2506_18150_gb300 import helrm as H
    ctx, p, sk, evk, sk_o, keys_o = env
    if z is None:
        z = np.random.default_rng(seed).uniform(-1, 1, p.n)
    m = ckks.encode_real(p, z, p.delta)
    ct = H.helrm_encrypt(ctx, evk, H.helrm_pt_import(ctx, m, level, p.delta), seed)
    ct_o = ckks.encrypt(p, keys_o, m, level, p.delta, seed)
    return ct, ct_o, z


def test_primes_and_roots_match_oracle(env):
    from paper_2506_18150_gb300 import helrm as H
    ctx, p = env[0], env[1]
    primes, psis = H.helrm_ctx_primes(ctx)
    assert primes == p.q + p.p
    assert psis == [p.psi[m] for m in p.q + p.p]
    assert H.helrm_ctx_dims(ctx)[:5] == [p.N, p.n, p.L, p.K, p.alpha]


@pytest.mark.parametrize("which", ["reduced", "full"])
def test_ntt_matches_oracle_evaluation(env, which):
    import torch

    from oracle import ring
    from paper_2506_18150_gb300 import helrm as H
    from paper_2506_18150_gb300 import synthetic as syn
    if which == "full":
        pr = syn.PARAMS["full"]
        ctx = gpu_ctx(pr)
        primes, psis = H.helrm_ctx_primes(ctx)
        log_n = pr["log_n"]
        pick = [0, 1, 20, 21, 23]                     # q_0 (60-bit), 40-bit, last q, two special primes
    else:
        ctx, p = env[0], env[1]
        primes, psis = H.helrm_ctx_primes(ctx)
        log_n = p.log_n
        pick = list(range(len(primes)))
    n = 1 << log_n
    rng = np.random.default_rng(7)
    brv = bitrev_perm(log_n)
    lo, hi = min(pick), max(pick)
    cnt = hi - lo + 1
    a = np.stack([rng.integers(0, primes[lo + i], n, dtype=np.uint64) for i in range(cnt)])
    a[0, :5] = 0
    a[-1, -3:] = np.uint64(primes[hi] - 1)                # edge residues
    dev = torch.from_numpy(a.view(np.int64).copy()).cuda()
    H.helrm_ntt(ctx, dev.data_ptr(), cnt, lo, False)
    H.helrm_ctx_synchronize(ctx)
    fwd = dev.cpu().numpy().view(np.uint64)
    for i in pick:
        l = i - lo
        want = ring.ntt(a[l], [primes[i]], [psis[i]])[0]
        assert np.array_equal(fwd[l], want[brv]), f"prime {i}"
    H.helrm_ntt(ctx, dev.data_ptr(), cnt, lo, True)
    H.helrm_ctx_synchronize(ctx)
    assert np.array_equal(dev.cpu().numpy().view(np.uint64), a)


@pytest.mark.parametrize("ept", ["4", "8"])
def test_ntt_both_thread_widths_full(ept, monkeypatch):
    """The N = 2^16 transform with 4 and with 8 elements per thread (the
    autotuner's radix-4 and radix-8 rounds; HELRM_NTT_EPT keeps one of them),
    at 1, 3 and 21 limbs per launch, against the oracle's evaluation."""
    import torch

    from oracle import ring
    from paper_2506_18150_gb300 import helrm as H
    from paper_2506_18150_gb300 import synthetic as syn
    monkeypatch.setenv("HELRM_NTT_EPT", ept)
    pr = syn.PARAMS["full"]
    ctx = gpu_ctx(pr)
    primes, psis = H.helrm_ctx_primes(ctx)
    tun = H.helrm_ctx_ntt_tuning(ctx)
    assert all(v[2] == int(ept) for v in tun.values())
    n = 1 << pr["log_n"]
    brv = bitrev_perm(pr["log_n"])
    rng = np.random.default_rng(11)
    for cnt in (1, 3, 21):
        a = np.stack([rng.integers(0, primes[1 + i], n, dtype=np.uint64) for i in range(cnt)])
        dev = torch.from_numpy(a.view(np.int64).copy()).cuda()
        H.helrm_ntt(ctx, dev.data_ptr(), cnt, 1, False)
        H.helrm_ctx_synchronize(ctx)
        fwd = dev.cpu().numpy().view(np.uint64)
        for l in sorted({0, cnt - 1}):
            want = ring.ntt(a[l], [primes[1 + l]], [psis[1 + l]])[0]
            assert np.array_equal(fwd[l], want[brv]), (cnt, l)
        H.helrm_ntt(ctx, dev.data_ptr(), cnt, 1, True)
        H.helrm_ctx_synchronize(ctx)
        assert np.array_equal(dev.cpu().numpy().view(np.uint64), a), cnt


def test_encryption_bit_exact(env):
    for level in [0, 2, 4]:
        ct, ct_o, _ = fresh(env, level, 1000 + level)
        assert_ct_equal(env[0], ct, ct_o)


def test_decrypt_matches_slots(env):
    from paper_2506_18150_gb300 import helrm as H
    ctx, p, sk = env[0], env[1], env[2]
    ct, ct_o, z = fresh(env, 3, 5)
    got = H.helrm_decrypt(ctx, sk, ct, p.n)
    assert np.max(np.abs(got - z)) < 1e-6
    got1 = H.helrm_decrypt(ctx, sk, ct, 3)                # direct (few-slot) decoder
    assert np.max(np.abs(got1 - z[:3])) < 1e-6


def test_encoder_within_one_unit_of_oracle(env):
    from oracle import ckks
    from paper_2506_18150_gb300 import helrm as H
    ctx, p = env[0], env[1]
    z = np.random.default_rng(11).uniform(-1, 1, p.n)
    pt = H.helrm_encode(ctx, z, 2, p.delta)
    got = H.helrm_pt_export(ctx, pt)
    want = ckks.encode_real(p, z, p.delta).astype(np.int64)
    d = np.abs(got - want)
    assert d.max() <= 1 and d.sum() <= max(8, p.N // 256)


def test_rescale_bit_exact(env):
    from oracle import ckks
    from paper_2506_18150_gb300 import helrm as H
    ctx, p = env[0], env[1]
    for level in [1, 4]:
        ct, ct_o, _ = fresh(env, level, 20 + level)
        assert_ct_equal(ctx, H.helrm_rescale(ctx, ct), ckks.rescale(p, ct_o))


@pytest.mark.parametrize("step", STEPS)
def test_rotation_bit_exact(env, step):
    from oracle import ckks
    from paper_2506_18150_gb300 import helrm as H
    ctx, p, sk, evk, sk_o, keys_o = env
    for level in [0, 4]:
        ct, ct_o, z = fresh(env, level, 30 + level)
        r = H.helrm_rotate(ctx, evk, ct, step)
        assert_ct_equal(ctx, r, ckks.rotate(p, keys_o, ct_o, step))
        assert np.max(np.abs(H.helrm_decrypt(ctx, sk, r, p.n) - np.roll(z, -step))) < 1e-6


def test_hoisted_rotation_bit_exact(env):
    from oracle import ckks
    from paper_2506_18150_gb300 import helrm as H
    ctx, p, sk, evk, sk_o, keys_o = env
    ct, ct_o, _ = fresh(env, 3, 44)
    outs = H.helrm_rotate_hoisted(ctx, evk, ct, STEPS + [0])
    want = ckks.rotate_hoisted(p, keys_o, ct_o, STEPS + [0])
    for s, o in zip(STEPS + [0], outs):
        assert_ct_equal(ctx, o, want[s])


def test_mul_add_sub_bit_exact(env):
    from oracle import ckks
    from paper_2506_18150_gb300 import helrm as H
    ctx, p, sk, evk, sk_o, keys_o = env
    a, a_o, x = fresh(env, 4, 50)
    b, b_o, y = fresh(env, 4, 51)
    assert_ct_equal(ctx, H.helrm_add(ctx, a, b), ckks.add(p, a_o, b_o))
    assert_ct_equal(ctx, H.helrm_sub(ctx, a, b), ckks.sub(p, a_o, b_o))
    c = H.helrm_mul(ctx, evk, a, b)
    assert_ct_equal(ctx, c, ckks.mul(p, keys_o, a_o, b_o))
    assert np.max(np.abs(H.helrm_decrypt(ctx, sk, c, p.n) - x * y)) < 1e-6
    sq = H.helrm_mul(ctx, evk, a, a)
    assert_ct_equal(ctx, sq, ckks.square(p, keys_o, a_o))
    m = ckks.encode_real(p, y, p.q[4])
    pt = H.helrm_pt_import(ctx, m, 4, float(p.q[4]))
    assert_ct_equal(ctx, H.helrm_mul_pt(ctx, a, pt), ckks.mul_pt(p, a_o, m, float(p.q[4])))
    md = ckks.encode_real(p, y, p.delta)
    assert_ct_equal(ctx, H.helrm_add_pt(ctx, a, H.helrm_pt_import(ctx, md, 4, p.delta)),
                    ckks.add_pt(p, a_o, md, p.delta))
    assert_ct_equal(ctx, H.helrm_drop_level(ctx, a, 1), ckks.drop_level(p, a_o, 1))


def test_import_export_round_trip_and_corruption(env):
    from paper_2506_18150_gb300 import helrm as H
    ctx, p = env[0], env[1]
    ct, ct_o, _ = fresh(env, 2, 60)
    back = import_ct(ctx, ct_o)
    assert_ct_equal(ctx, back, ct_o)
    bad = np.stack([ct_o.c0, ct_o.c1]).copy()
    bad[1, 2, 17] = np.uint64(p.q[2])                    # residue == its prime
    with pytest.raises(H.HelrmError) as e:
        H.helrm_ct_import(ctx, bad, 2, p.delta)
    assert e.value.name == "HELRM_E_INVAL"


def test_error_paths(env):
    from paper_2506_18150_gb300 import helrm as H
    ctx, p, sk, evk = env[0], env[1], env[2], env[3]
    a, _, _ = fresh(env, 3, 70)
    b, _, _ = fresh(env, 2, 71)
    with pytest.raises(H.HelrmError) as e:
        H.helrm_rotate(ctx, evk, a, 2)                    # no key for step 2
    assert e.value.name == "HELRM_E_NOKEY"
    with pytest.raises(H.HelrmError) as e:
        H.helrm_add(ctx, a, b)
    assert e.value.name == "HELRM_E_LEVEL"
    c = H.helrm_rescale(ctx, H.helrm_mul_pt(ctx, a, H.helrm_pt_import(ctx, np.ones(p.N, np.int64), 3, 3.0)))
    with pytest.raises(H.HelrmError) as e:
        H.helrm_add(ctx, c, H.helrm_drop_level(ctx, a, 2))
    assert e.value.name == "HELRM_E_SCALE"
    z0, _, _ = fresh(env, 0, 72)
    with pytest.raises(H.HelrmError) as e:
        H.helrm_rescale(ctx, z0)
    assert e.value.name == "HELRM_E_LEVEL"


def test_memory_cap_gives_nomem(env):
    from paper_2506_18150_gb300 import helrm as H
    ctx, p = env[0], env[1]
    a, _, _ = fresh(env, 4, 80)
    used = H.helrm_ctx_memory_in_use(ctx)
    H.helrm_ctx_set_memory_cap(ctx, used + 1024)
    try:
        with pytest.raises(H.HelrmError) as e:
            H.helrm_add(ctx, a, a)
        assert e.value.name == "HELRM_E_NOMEM"
    finally:
        H.helrm_ctx_set_memory_cap(ctx, 0)
    H.helrm_add(ctx, a, a)                                 # usable again


def test_bounded_device_wait_reports_timeout_and_context_survives(env):
    """A device-side wait that never completes ends after its poll limit with
    HELRM_E_TIMEOUT (no hang, no trap), and the context keeps working."""
    from paper_2506_18150_gb300 import helrm as H
    ctx, p, sk, evk = env[0], env[1], env[2], env[3]
    for polls in (1, 1000):
        with pytest.raises(H.HelrmError) as e:
            H.helrm_ctx_wait_selftest(ctx, polls)
        assert e.value.name == "HELRM_E_TIMEOUT"
    with pytest.raises(H.HelrmError) as e:
        H.helrm_ctx_wait_selftest(ctx, 0)
    assert e.value.name == "HELRM_E_INVAL"
    a, _, _ = fresh(env, 3, 71)                   # the context still encrypts and rescales
    H.helrm_rescale(ctx, a)
    H.helrm_ctx_synchronize(ctx)
