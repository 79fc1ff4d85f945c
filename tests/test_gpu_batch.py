"""Lockstep batched inference (helrm_batch_create / helrm_infer_batch): many
clients' queries of one model run through every step together.  The server
arithmetic is deterministic integer math, so each query's logit ciphertext
must be bit-identical to the one the one-query path gives it alone -- and,
with the oracle's integer plaintexts and keys, bit-identical to the oracle's.
The decrypted logits must stay within 1e-3 of the FP64 cleartext DLRM."""
import numpy as np
import pytest

from helpers import assert_ct_equal, export_ct, gpu_ctx, oracle_params

pytestmark = pytest.mark.gpu


def _same_ct(ctx, a, b):
    ca, la, sa = export_ct(ctx, a)
    cb, lb, sb = export_ct(ctx, b)
    assert la == lb and sa == sb
    assert np.array_equal(ca, cb), "ciphertexts differ"


@pytest.mark.parametrize("interaction", ["dot", "concat"])
def test_batch_matches_single_and_oracle_reduced(interaction):
    """N = 2^13, UCI-shaped model, three queries from two clients (client 0
    twice).  Client 0's keys are the oracle's (same seed), so its two batched
    logits are also compared with the oracle's ciphertexts bit for bit."""
    from oracle import ckks, dlrm
    from paper_2506_18150_gb300 import helrm as H
    from paper_2506_18150_gb300 import synthetic as syn
    pr = syn.reduced_params(13, 9)
    spec = syn.uci_spec(0, interaction)
    w = syn.make_weights(spec, 0)
    p = oracle_params(pr)
    comp = dlrm.compile_model(p, spec, w)
    ctx = gpu_ctx(pr)
    model = H.helrm_model_create(ctx, spec, w)
    H.helrm_model_import_plaintexts(ctx, model, np.stack([np.asarray(x, dtype=np.int64) for x in comp.plaintexts()]))
    steps = H.helrm_model_rotations(ctx, model)
    keys = [H.helrm_keygen(ctx, s, steps) for s in (1, 2)]
    _, keys_o = ckks.keygen(p, 1, rot_steps=comp.rotation_steps())
    owner = [0, 1, 0]
    dense, idx = syn.make_queries(spec, 3, seed=5)
    cd, cs, outs_o = [], [], {}
    for q in range(3):
        xd, xs = dlrm.query_slots(p, comp, dense[q], idx[q])
        md, ms = ckks.encode_real(p, xd, p.delta), ckks.encode_real(p, xs, p.delta)
        evk = keys[owner[q]][1]
        cd.append(H.helrm_encrypt(ctx, evk, H.helrm_pt_import(ctx, md, comp.lvl_dense, p.delta), 100 + 2 * q))
        cs.append(H.helrm_encrypt(ctx, evk, H.helrm_pt_import(ctx, ms, comp.lvl_sel, p.delta), 101 + 2 * q))
        if owner[q] == 0:
            cd_o = ckks.encrypt(p, keys_o, md, comp.lvl_dense, p.delta, 100 + 2 * q)
            cs_o = ckks.encrypt(p, keys_o, ms, comp.lvl_sel, p.delta, 101 + 2 * q)
            outs_o[q] = dlrm.infer(p, keys_o, comp, cd_o, cs_o)
    batch = H.helrm_batch_create(ctx, model, [keys[o][1] for o in owner])
    got = H.helrm_infer_batch(ctx, batch, cd, cs)
    for q in range(3):
        alone = H.helrm_infer(ctx, keys[owner[q]][1], model, cd[q], cs[q])
        _same_ct(ctx, got[q], alone)
        if q in outs_o:
            assert_ct_equal(ctx, got[q], outs_o[q])
        ref = dlrm.dlrm_cleartext(spec, w, dense[q], idx[q])[0]
        lg, _ = H.helrm_decrypt_logit(ctx, keys[owner[q]][0], got[q])
        assert abs(lg - ref) < 1e-3, (q, lg, ref)


def _full_batch(spec_fn, n_clients, owner, seed):
    import torch

    from oracle import dlrm
    from paper_2506_18150_gb300 import helrm as H
    from paper_2506_18150_gb300 import synthetic as syn
    spec = spec_fn(0)
    w = syn.make_weights(spec, 0)
    ctx = gpu_ctx(syn.PARAMS["full"])
    model = H.helrm_model_create(ctx, spec, w)
    steps = H.helrm_model_rotations(ctx, model)
    keys = [H.helrm_keygen(ctx, 50 + c, steps) for c in range(n_clients)]
    n = len(owner)
    dense, idx = syn.make_queries(spec, n, seed=seed)
    batch = H.helrm_batch_create(ctx, model, [keys[o][1] for o in owner])
    d_dense = torch.tensor(dense, dtype=torch.float64, device="cuda")
    d_idx = torch.tensor(idx.astype(np.int64), dtype=torch.int64, device="cuda")
    d_lg = torch.zeros(n, dtype=torch.float64, device="cuda")
    H.helrm_infer_batch_e2e_device(ctx, batch, [keys[o][0] for o in owner], d_dense.data_ptr(), d_idx.data_ptr(),
                                   77, d_lg.data_ptr())
    lg = d_lg.cpu().numpy()
    for q in range(n):
        sk, evk = keys[owner[q]]
        # the same query alone through the one-query protocol, same seed
        cd, cs = H.helrm_encrypt_query(ctx, evk, model, dense[q], idx[q], 77 + 2 * q)
        alone, _ = H.helrm_decrypt_logit(ctx, sk, H.helrm_infer(ctx, evk, model, cd, cs))
        assert lg[q] == alone, (q, lg[q], alone)
        ref = dlrm.dlrm_cleartext(spec, w, dense[q], idx[q])[0]
        assert abs(lg[q] - ref) < 1e-3, (q, lg[q], ref)


def test_batch_full_uci():
    """UCI-shaped model at N = 2^16: five queries, three clients, uneven ownership."""
    from paper_2506_18150_gb300 import synthetic as syn
    _full_batch(syn.uci_spec, 3, [0, 1, 2, 1, 1], 41)


def test_batch_full_criteo():
    """Criteo-shaped model at N = 2^16: three queries of two clients."""
    from paper_2506_18150_gb300 import synthetic as syn
    _full_batch(syn.criteo_spec, 2, [1, 0, 1], 43)


def test_batch_errors():
    from paper_2506_18150_gb300 import helrm as H
    from paper_2506_18150_gb300 import synthetic as syn
    pr = syn.reduced_params(13, 9)
    spec = syn.uci_spec(0)
    ctx = gpu_ctx(pr)
    model = H.helrm_model_create(ctx, spec, syn.make_weights(spec, 0))
    sk, evk = H.helrm_keygen(ctx, 3, [1, 2])            # lacks most of the model's rotations
    with pytest.raises(H.HelrmError) as e:
        H.helrm_batch_create(ctx, model, [evk])
    assert e.value.name == "HELRM_E_NOKEY"
    sk, evk = H.helrm_keygen(ctx, 3, H.helrm_model_rotations(ctx, model))
    batch = H.helrm_batch_create(ctx, model, [evk, evk])
    dense, idx = syn.make_queries(spec, 2, seed=1)
    cts = [H.helrm_encrypt_query(ctx, evk, model, dense[q], idx[q], 9 + 2 * q) for q in range(2)]
    with pytest.raises(H.HelrmError) as e:               # dense and selector swapped: wrong levels
        H.helrm_infer_batch(ctx, batch, [c[1] for c in cts], [c[0] for c in cts])
    assert e.value.name == "HELRM_E_LEVEL"


def test_model_keygen_truncated_keys_give_identical_logits():
    """helrm_model_keygen: each key generated only up to the level the model
    uses it at.  The key values are the full keys' restrictions, so the logit
    ciphertexts are bit-identical to those under full keys, in less memory; a
    truncated key used above its level is refused (HELRM_E_NOKEY)."""
    from paper_2506_18150_gb300 import helrm as H
    from paper_2506_18150_gb300 import synthetic as syn
    pr = syn.reduced_params(13, 12)          # three spare levels above the model's
    spec = syn.uci_spec(0)
    ctx = gpu_ctx(pr)
    model = H.helrm_model_create(ctx, spec, syn.make_weights(spec, 0))
    steps = H.helrm_model_rotations(ctx, model)
    sk_f, evk_f = H.helrm_keygen(ctx, 9, steps)
    sk_t, evk_t = H.helrm_model_keygen(ctx, model, 9)
    assert H.helrm_evk_bytes(ctx, evk_t) < 0.6 * H.helrm_evk_bytes(ctx, evk_f)
    dense, idx = syn.make_queries(spec, 2, seed=4)
    for q in range(2):
        cd, cs = H.helrm_encrypt_query(ctx, evk_f, model, dense[q], idx[q], 50 + 2 * q)
        a = H.helrm_infer(ctx, evk_f, model, cd, cs)
        b = H.helrm_infer(ctx, evk_t, model, cd, cs)
        _same_ct(ctx, a, b)
        batch = H.helrm_batch_create(ctx, model, [evk_t])
        _same_ct(ctx, a, H.helrm_infer_batch(ctx, batch, [cd], [cs])[0])
    top = H.helrm_encrypt(ctx, evk_t, H.helrm_encode(ctx, np.ones(8), 12, 2.0**40), 3)
    with pytest.raises(H.HelrmError) as e:
        H.helrm_rotate(ctx, evk_t, top, steps[-1])
    assert e.value.name == "HELRM_E_NOKEY"


def test_batch_graph_replay_matches_eager():
    """helrm_batch_set_graph: the batch's server path captured as a CUDA graph
    and replayed on new inputs gives the eager path's ciphertexts bit for bit
    (first call: capture; second and third: replays with other queries)."""
    from paper_2506_18150_gb300 import helrm as H
    from paper_2506_18150_gb300 import synthetic as syn
    pr = syn.reduced_params(13, 9)
    spec = syn.uci_spec(0)
    ctx = gpu_ctx(pr)
    model = H.helrm_model_create(ctx, spec, syn.make_weights(spec, 0))
    keys = [H.helrm_model_keygen(ctx, model, 70 + c) for c in range(2)]
    owner = [0, 1, 1]
    eager = H.helrm_batch_create(ctx, model, [keys[o][1] for o in owner])
    graph = H.helrm_batch_create(ctx, model, [keys[o][1] for o in owner])
    H.helrm_batch_set_graph(ctx, graph, True)
    for call in range(3):
        dense, idx = syn.make_queries(spec, 3, seed=80 + call)
        cts = [H.helrm_encrypt_query(ctx, keys[owner[q]][1], model, dense[q], idx[q], 500 + 10 * call + 2 * q)
               for q in range(3)]
        a = H.helrm_infer_batch(ctx, eager, [c[0] for c in cts], [c[1] for c in cts])
        b = H.helrm_infer_batch(ctx, graph, [c[0] for c in cts], [c[1] for c in cts])
        for q in range(3):
            _same_ct(ctx, a[q], b[q])


def test_batch_e2e_host_buffers_with_graph():
    """helrm_infer_batch_e2e from host buffers, the batch's server path
    replayed as a CUDA graph: the logits equal helrm_infer_e2e's for the same
    queries and seeds (twice: the capture, then a replay)."""
    from paper_2506_18150_gb300 import helrm as H
    from paper_2506_18150_gb300 import synthetic as syn
    pr = syn.reduced_params(13, 9)
    spec = syn.uci_spec(0)
    ctx = gpu_ctx(pr)
    model = H.helrm_model_create(ctx, spec, syn.make_weights(spec, 0))
    sk, evk = H.helrm_model_keygen(ctx, model, 90)
    batch = H.helrm_batch_create(ctx, model, [evk, evk])
    H.helrm_batch_set_graph(ctx, batch, True)
    for call in range(2):
        dense, idx = syn.make_queries(spec, 2, seed=95 + call)
        want, _ = H.helrm_infer_e2e(ctx, sk, evk, model, dense, idx, 300 + call)
        got = H.helrm_infer_batch_e2e(ctx, batch, [sk, sk], dense, idx, 300 + call)
        assert list(got) == list(want)
