"""The binding frees a context only after every handle that depends on it
(the library requires that order): also when the cyclic garbage collector
finalises a context and its handles together, in no particular order (a
traceback kept by pytest.raises holds such a cycle).  Runs without the
library: the free call is replaced by a recorder."""
import gc

import pytest


@pytest.fixture
def freed(monkeypatch):
    from paper_2506_18150_gb300 import helrm as H
    log = []

    class Recorder:
        def helrm_free(self, p):
            log.append(p.value)

    monkeypatch.setattr(H, "_lib", Recorder())
    return log


def test_context_outlives_its_handles_in_a_cycle(freed):
    from paper_2506_18150_gb300 import helrm as H
    ctx = H.Context(1)
    a = H.Handle(2, ctx)
    b = H.Handle(3, (ctx, a))            # a batch-like handle: its context inside a tuple
    c = H.Borrowed(4, a)                 # owned by a: never freed by the binding
    box = [ctx, a, b, c]
    box.append(box)                      # a reference cycle holding all of them
    del ctx, a, b, c, box
    gc.collect()
    assert sorted(freed[:-1]) == [2, 3] and freed[-1] == 1


def test_context_freed_at_once_without_handles(freed):
    from paper_2506_18150_gb300 import helrm as H
    ctx = H.Context(7)
    h = H.Handle(8, ctx)
    del h
    assert freed == [8]
    del ctx
    assert freed == [8, 7]


def test_context_dropped_first_waits_for_the_last_handle(freed):
    from paper_2506_18150_gb300 import helrm as H
    ctx = H.Context(5)
    h = H.Handle(6, ctx)
    ctx.__del__()                        # the context's finaliser runs first
    assert freed == []
    del h
    assert freed == [6, 5]
