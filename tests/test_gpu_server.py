"""Continuous-batching server: every result equals the same graph embedded alone (and
the oracle), the memory budget is never exceeded, oversized requests are refused, queued
requests can be cancelled, released memory is returned."""
import numpy as np
import pytest

import oracle
from synth import batch_graph, batch_specs

from gpu_util import assert_z_matches, dev_graph

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
ALL = 7


@pytest.fixture(scope="module")
def gee():
    import paper_2406_03726_gb300 as gee
    gee.lib()
    return gee


def mix(G, seed, n_range=(100, 8000), d_range=(5.0, 80.0)):
    return [batch_graph(s) for s in batch_specs(G, seed=seed, n_range=n_range, d_range=d_range)]


def solo(gee, g):
    s, d, w, y = dev_graph(g)
    Z = gee.embed(s, d, w, g.N, y, g.K, ALL)
    torch.cuda.synchronize()
    return Z.cpu().numpy()


def test_server_results_equal_solo_and_oracle(gee):
    graphs = mix(60, seed=51)
    srv = gee.Server(1 << 30, ALL)
    tickets = [srv.submit(g.src, g.dst, g.w, g.labels, g.N, g.K) for g in graphs]
    for g, t in zip(graphs, tickets):
        z, st, lat = srv.poll(t, wait=True)
        assert st == 0 and lat >= 0
        Z = srv.fetch(t)
        assert np.array_equal(Z, solo(gee, g)), g.name            # same alone and in the mix
        assert_z_matches(Z.astype(np.float64), oracle.embed_graph(g, ALL), what=g.name)
        srv.release(t)
    s = srv.stats()
    assert s["completed"] == len(graphs) and s["bytes_in_use"] == 0
    assert s["peak_bytes_in_use"] <= s["pool_bytes"] and s["last_error"] == 0
    srv.close()


def test_server_small_budget_admits_as_memory_frees(gee):
    graphs = mix(30, seed=52, n_range=(2000, 6000), d_range=(40.0, 80.0))
    need = max(gee.gee_workspace_size(g.E, g.N, g.K, True, gee.make_opts(ALL)) + g.E * 12 + g.N * (4 + 4 * g.K)
               for g in graphs)
    budget = 3 * need + (8 << 20)                  # room for about two requests in flight
    srv = gee.Server(budget, ALL, streams=2)
    tickets = [srv.submit(g.src, g.dst, g.w, g.labels, g.N, g.K) for g in graphs]
    for g, t in zip(graphs, tickets):
        srv.poll(t, wait=True)
        Z = srv.fetch(t)
        assert np.array_equal(Z, solo(gee, g))
        srv.release(t)                             # frees memory for the requests still queued
    s = srv.stats()
    assert s["completed"] == len(graphs)
    assert s["peak_bytes_in_use"] <= budget and s["bytes_in_use"] == 0
    srv.close()


def test_server_refuses_request_larger_than_budget(gee):
    g = mix(1, seed=53, n_range=(20000, 20000), d_range=(150.0, 150.0))[0]
    srv = gee.Server(8 << 20, ALL)
    with pytest.raises(gee.GeeError) as e:
        srv.submit(g.src, g.dst, g.w, g.labels, g.N, g.K)
    assert e.value.code == gee.ERR_NOMEM
    srv.close()


def test_server_cancel_and_state_errors(gee):
    graphs = mix(6, seed=54, n_range=(3000, 3000), d_range=(60.0, 60.0))
    need = gee.gee_workspace_size(graphs[0].E, graphs[0].N, graphs[0].K, True, gee.make_opts(ALL)) \
        + graphs[0].E * 12 + graphs[0].N * (4 + 4 * graphs[0].K)
    srv = gee.Server(need + need // 2 + (4 << 20), ALL, streams=1)     # one request at a time
    tickets = [srv.submit(g.src, g.dst, g.w, g.labels, g.N, g.K) for g in graphs]
    # the last request is still queued behind the first (not released yet): cancel it
    assert srv.cancel(tickets[-1]) == 0
    assert gee.gee_server_poll(srv.handle, tickets[-1])[0] == gee.ERR_STATE
    for g, t in zip(graphs[:-1], tickets[:-1]):
        srv.poll(t, wait=True)
        assert srv.cancel(t) == gee.ERR_STATE          # too late to cancel
        assert np.array_equal(srv.fetch(t), solo(gee, g))
        srv.release(t)
    assert gee.gee_server_release(srv.handle, tickets[0]) == gee.ERR_STATE   # already released
    assert srv.stats()["bytes_in_use"] == 0
    srv.close()


def test_server_replays_a_seeded_poisson_trace(gee):
    """Requests arrive on a seeded Poisson trace while earlier ones run (pageable and pinned
    host inputs mixed, a tight budget so admission waits for memory): every result equals
    the same graph embedded alone, bit for bit."""
    import threading
    import time
    graphs = mix(48, seed=53, n_range=(200, 20000), d_range=(5.0, 120.0))
    rng = np.random.default_rng(54)
    gaps = rng.exponential(0.002, len(graphs))           # about 500 requests per second
    host = []
    for i, g in enumerate(graphs):
        if i % 2:  # pinned inputs for every second request
            pin = [torch.from_numpy(a).pin_memory().numpy() for a in (g.src, g.dst, g.w, g.labels)]
            host.append(tuple(pin))
        else:
            host.append((g.src, g.dst, g.w, g.labels))
    need = max(8 * g.E * 4 + g.N * g.K * 4 for g in graphs)
    srv = gee.Server(max(64 << 20, 6 * need), ALL, max_batch=16, streams=2)
    tickets = [None] * len(graphs)

    def submitter():
        for i, (g, h) in enumerate(zip(graphs, host)):
            time.sleep(gaps[i])
            tickets[i] = srv.submit(h[0], h[1], h[2], h[3], g.N, g.K)

    th = threading.Thread(target=submitter)
    th.start()
    for i, g in enumerate(graphs):
        while tickets[i] is None:
            time.sleep(0.0005)
        z, st, lat = srv.poll(tickets[i], wait=True)
        assert st == 0
        assert np.array_equal(srv.fetch(tickets[i]), solo(gee, g)), g.name
        srv.release(tickets[i])
    th.join()
    s = srv.stats()
    assert s["completed"] == len(graphs) and s["bytes_in_use"] == 0 and s["last_error"] == 0
    assert s["peak_bytes_in_use"] <= s["pool_bytes"] and s["launches"] >= 2
    srv.close()
