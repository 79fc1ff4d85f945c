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
