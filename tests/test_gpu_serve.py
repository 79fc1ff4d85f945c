"""The serving loop (helrm_server_*): requests that arrive while others are
on the GPU join new batches on free slots, and batches of different models
run concurrently.  The server arithmetic is deterministic integer math, so
every request's encrypted logit must be bit-identical to the one
helrm_infer gives that request alone, whatever it was batched with."""
import numpy as np
import pytest

from helpers import export_ct, gpu_ctx

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pool():
    """N = 2^13, two UCI-shaped models with different table sets (seeds 0
    and 1), three clients of the first and two of the second, 14 requests."""
    from paper_2506_18150_gb300 import helrm as H
    from paper_2506_18150_gb300 import synthetic as syn
    pr = syn.reduced_params(13, 9)
    ctx = gpu_ctx(pr)
    specs = [syn.uci_spec(0), syn.uci_spec(1)]
    models = [H.helrm_model_create(ctx, s, syn.make_weights(s, 0)) for s in specs]
    owner_model = [0, 0, 0, 1, 1]
    keys = [H.helrm_keygen(ctx, 200 + c, H.helrm_model_rotations(ctx, models[m])) for c, m in enumerate(owner_model)]
    rng = np.random.default_rng(7)
    n = 14
    client = rng.integers(0, len(owner_model), n)
    arrival = np.sort(np.concatenate([np.zeros(5), rng.uniform(0, 0.01, n - 5)]))   # a burst, then a trickle
    cts = []
    for r in range(n):
        m = owner_model[client[r]]
        dense, idx = syn.make_queries(specs[m], 1, seed=300 + r)
        cts.append(H.helrm_encrypt_query(ctx, keys[client[r]][1], models[m], dense[0], idx[0], 1000 + 2 * r))
    alone = []
    for r in range(n):
        m = owner_model[client[r]]
        alone.append(export_ct(ctx, H.helrm_infer(ctx, keys[client[r]][1], models[m], *cts[r]))[0])
    return dict(ctx=ctx, models=models, owner_model=owner_model, keys=keys, client=client, arrival=arrival,
                cts=cts, alone=alone)


def _serve(p, n_slots, max_batch, budget=0):
    from paper_2506_18150_gb300 import helrm as H
    ctx = p["ctx"]
    srv = H.helrm_server_create(ctx, n_slots, max_batch, budget)
    for c, m in enumerate(p["owner_model"]):
        assert H.helrm_server_add_client(ctx, srv, p["models"][m], p["keys"][c][1]) == c
    outs, lat, st = H.helrm_server_run(ctx, srv, p["arrival"], p["client"], [c[0] for c in p["cts"]],
                                       [c[1] for c in p["cts"]])
    for r, o in enumerate(outs):
        got = export_ct(ctx, o)[0]
        assert np.array_equal(got, p["alone"][r]), f"request {r} differs from its one-query result"
    assert np.all(lat > 0) and st["n_batches"] >= 1
    return lat, st


def test_served_results_match_alone_with_batching(pool):
    lat, st = _serve(pool, n_slots=2, max_batch=4)
    assert st["max_batch"] > 1, "the burst should have been batched"
    assert st["n_batches"] < len(pool["arrival"])
    assert st["p50_ms"] <= st["p99_ms"] <= st["max_ms"]


def test_plain_one_request_at_a_time_path(pool):
    _, st = _serve(pool, n_slots=1, max_batch=1)
    assert st["max_batch"] == 1 and st["n_batches"] == len(pool["arrival"]) and st["max_inflight"] == 1


def test_memory_budget_limits_batches(pool):
    _, st = _serve(pool, n_slots=2, max_batch=8, budget=1)   # room for nothing: one request at a time
    assert st["max_batch"] == 1 and st["max_inflight"] == 1


def test_server_argument_errors(pool):
    from paper_2506_18150_gb300 import helrm as H
    ctx = pool["ctx"]
    with pytest.raises(H.HelrmError) as e:
        H.helrm_server_create(ctx, 0, 4)
    assert e.value.name == "HELRM_E_INVAL"
    srv = H.helrm_server_create(ctx, 1, 2)
    H.helrm_server_add_client(ctx, srv, pool["models"][0], pool["keys"][0][1])
    with pytest.raises(H.HelrmError) as e:   # client 3 was never registered
        H.helrm_server_run(ctx, srv, [0.0], [3], [pool["cts"][0][0]], [pool["cts"][0][1]])
    assert e.value.name == "HELRM_E_INVAL"
    with pytest.raises(H.HelrmError) as e:   # arrivals out of order
        H.helrm_server_run(ctx, srv, [0.5, 0.1], [0, 0], [pool["cts"][0][0]] * 2, [pool["cts"][0][1]] * 2)
    assert e.value.name == "HELRM_E_INVAL"


def _oracle_served(ctx, srv, arrival, client, cts):
    from paper_2506_18150_gb300 import helrm as H
    outs, lat, st = H.helrm_server_run(ctx, srv, arrival, client, [c[0] for c in cts], [c[1] for c in cts])
    return [export_ct(ctx, o)[0] for o in outs], st


def test_served_logits_bit_exact_against_oracle():
    """A burst of 4 UCI-shaped requests of one client at N = 2^13, served in
    one batch, with the oracle's integer plaintexts in the model and the
    query ciphertexts encrypted from the oracle's encodings with the same
    seeds: the served logit ciphertexts of two requests equal the oracle's
    dlrm.infer word for word (the others equal them by the one-query check)."""
    from helpers import oracle_keys_pool, oracle_params
    from oracle import ckks, dlrm
    from paper_2506_18150_gb300 import helrm as H
    from paper_2506_18150_gb300 import synthetic as syn
    pr = syn.reduced_params(13, 9)
    p = oracle_params(pr)
    spec = syn.uci_spec(0)
    w = syn.make_weights(spec, 0)
    c = dlrm.compile_model(p, spec, w)
    _, keys_o = oracle_keys_pool(pr, 41, c.rotation_steps())     # the spawn pool starts before the GPU work
    ctx = gpu_ctx(pr)
    model = H.helrm_model_create(ctx, spec, w)
    H.helrm_model_import_plaintexts(ctx, model, np.stack([np.asarray(x, dtype=np.int64) for x in c.plaintexts()]))
    _, evk = H.helrm_keygen(ctx, 41, H.helrm_model_rotations(ctx, model))
    dense, idx = syn.make_queries(spec, 4, seed=71)
    cts, want = [], []
    for q in range(4):
        xd, xs = dlrm.query_slots(p, c, dense[q], idx[q])
        md, ms = ckks.encode_real(p, xd, p.delta), ckks.encode_real(p, xs, p.delta)
        cts.append((H.helrm_encrypt(ctx, evk, H.helrm_pt_import(ctx, md, c.lvl_dense, p.delta), 500 + 2 * q),
                    H.helrm_encrypt(ctx, evk, H.helrm_pt_import(ctx, ms, c.lvl_sel, p.delta), 501 + 2 * q)))
        if q < 2:
            want.append(dlrm.infer(p, keys_o, c, ckks.encrypt(p, keys_o, md, c.lvl_dense, p.delta, 500 + 2 * q),
                                   ckks.encrypt(p, keys_o, ms, c.lvl_sel, p.delta, 501 + 2 * q)))
    srv = H.helrm_server_create(ctx, 2, 4, 0)
    H.helrm_server_add_client(ctx, srv, model, evk)
    got, st = _oracle_served(ctx, srv, np.zeros(4), np.zeros(4, dtype=np.uint32), cts)
    assert st["max_batch"] > 1, "the burst should have been batched"
    for q in range(2):
        assert np.array_equal(got[q][0], want[q].c0) and np.array_equal(got[q][1], want[q].c1), \
            f"served request {q} differs from the oracle"
    for q in range(4):
        alone = export_ct(ctx, H.helrm_infer(ctx, evk, model, *cts[q]))[0]
        assert np.array_equal(got[q], alone), f"served request {q} differs from its one-query result"


def test_served_multi_ciphertext_selectors():
    """The wide DLRM (a 727-slot selector: two ciphertexts at N = 2^10) served
    to two clients with batching: each request brings its two selector
    ciphertexts; every served logit equals helrm_infer_multi alone, and two
    equal the oracle's word for word."""
    from helpers import oracle_params
    from oracle import ckks, dlrm
    from paper_2506_18150_gb300 import helrm as H
    from paper_2506_18150_gb300 import synthetic as syn
    pr = syn.reduced_params(10, 5)
    p = oracle_params(pr)
    spec = syn.wide_spec()
    w = syn.make_weights(spec, 0)
    c = dlrm.compile_model(p, spec, w)
    ctx = gpu_ctx(pr)
    model = H.helrm_model_create(ctx, spec, w)
    assert H.helrm_model_info(ctx, model)["n_sel"] == c.n_sel() == 2
    H.helrm_model_import_plaintexts(ctx, model, np.stack([np.asarray(x, dtype=np.int64) for x in c.plaintexts()]))
    steps = H.helrm_model_rotations(ctx, model)
    keys = [H.helrm_keygen(ctx, 80 + k, steps)[1] for k in range(2)]
    keys_o = [ckks.keygen(p, 80 + k, rot_steps=steps)[1] for k in range(2)]
    dense, idx = syn.make_queries(spec, 6, seed=9)
    client = np.array([0, 1, 0, 1, 1, 0], dtype=np.uint32)
    arrival = np.array([0.0, 0.0, 0.0, 0.001, 0.002, 0.003])
    cts, want = [], {}
    for q in range(6):
        xd, xs = dlrm.query_slots(p, c, dense[q], idx[q])
        md = ckks.encode_real(p, xd, p.delta)
        ms = [ckks.encode_real(p, x, p.delta) for x in xs]
        ev = keys[client[q]]
        cd = H.helrm_encrypt(ctx, ev, H.helrm_pt_import(ctx, md, c.lvl_dense, p.delta), 600 + 3 * q)
        cs = [H.helrm_encrypt(ctx, ev, H.helrm_pt_import(ctx, m, c.lvl_sel, p.delta), 601 + 3 * q + k)
              for k, m in enumerate(ms)]
        cts.append((cd, cs))
        if q in (1, 2):
            ko = keys_o[client[q]]
            want[q] = dlrm.infer(p, ko, c, ckks.encrypt(p, ko, md, c.lvl_dense, p.delta, 600 + 3 * q),
                                 [ckks.encrypt(p, ko, m, c.lvl_sel, p.delta, 601 + 3 * q + k) for k, m in enumerate(ms)])
    srv = H.helrm_server_create(ctx, 2, 4, 0)
    for k in range(2):
        assert H.helrm_server_add_client(ctx, srv, model, keys[k]) == k
    got, st = _oracle_served(ctx, srv, arrival, client, cts)
    assert st["n_batches"] < 6 and st["max_batch"] > 1
    for q in range(6):
        alone = export_ct(ctx, H.helrm_infer_multi(ctx, keys[client[q]], model, *cts[q]))[0]
        assert np.array_equal(got[q], alone), f"served request {q} differs from its one-query result"
    for q, y in want.items():
        assert np.array_equal(got[q][0], y.c0) and np.array_equal(got[q][1], y.c1), \
            f"served request {q} differs from the oracle"
