"""The continuous-batching server: every request gets the same result alone
and in the mix (bit for bit: the same groups of the same particles make the
same decisions in the same order), matches tpm_compute_forces within the FP32
tolerance, and the HBM budget forces evictions without changing results."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


def rel(a, b):
    return np.linalg.norm(a - b, axis=1) / np.maximum(np.linalg.norm(b, axis=1), 1e-300)


@pytest.fixture(scope="module")
def setup():
    import torch

    import paper_1909_04667_gb300 as tpm
    from paper_1909_04667_gb300.serve import ServeRequest

    cat = W.serving_catalogue(6, 11, nmin=2000, nmax=40000)
    parts = {s.sid: s.particles() for s in cat}

    def source(sid):
        pos, mass = parts[sid]
        s = cat[sid]
        return pos, mass, tpm.BuildParams(G=1.0, h=s.h, shift=tuple(W.root_shift(s.seed)), leaf_bucket=8)

    rng = np.random.default_rng(4)
    reqs = []
    for k in range(24):
        sid = int(rng.integers(0, len(cat)))
        n = cat[sid].n
        m = max(1, int(n * rng.uniform(0.01, 1.0)))
        reqs.append(ServeRequest(k, sid, rng.choice(n, m, replace=False).astype(np.int32), arrival=0.002 * k))
    return tpm, torch, cat, source, reqs


def fresh(reqs):
    from paper_1909_04667_gb300.serve import ServeRequest

    return [ServeRequest(r.rid, r.sid, r.ids.copy(), r.arrival) for r in reqs]


def test_alone_equals_mix_and_matches_compute_forces(setup):
    tpm, torch, cat, source, reqs = setup
    from paper_1909_04667_gb300.serve import ForceServer

    ctx = tpm.Context(0)
    srv = ForceServer(ctx, source, max_round_ids=1 << 18, max_round_requests=64, policy="bh")
    mixed = srv.serve(fresh(reqs), realtime=False)
    assert max(len(r.ids) for r in reqs) < (1 << 18)
    for r in fresh(reqs):
        alone = srv.serve([r], realtime=False)[0]
        m = next(x for x in mixed if x.rid == r.rid)
        np.testing.assert_array_equal(alone.acc, m.acc)
        np.testing.assert_array_equal(alone.n_int, m.n_int)
    srv.close()
    # and each matches a direct tpm_compute_forces call on the same tree
    for m in mixed[:6]:
        pos, mass, bp = source(m.sid)
        s = ctx.build_tree(pos, mass, bp)
        a, p, n = s.compute_forces(active_ids=m.ids, fp=tpm.ForceParams(theta=0.5))
        e = rel(m.acc.astype(np.float64), a.cpu().numpy().astype(np.float64))
        same = m.n_int == n.cpu().numpy()
        assert same.mean() >= 0.995 and np.percentile(e[same], 99) < 2e-5
        s.release()
    ctx.close()


def test_budget_evictions_keep_results(setup):
    tpm, torch, cat, source, _ = setup
    from paper_1909_04667_gb300.serve import ForceServer, ServeRequest, serve_per_request

    # two passes over the systems in increasing size: the largest tree is
    # built while the five smaller ones are resident
    rng = np.random.default_rng(9)
    order = sorted(range(len(cat)), key=lambda sid: cat[sid].n)
    reqs = []
    for sid in order * 2:
        n = cat[sid].n
        reqs.append(ServeRequest(len(reqs), sid, rng.choice(n, max(1, n // 3), replace=False).astype(np.int32),
                                 arrival=0.002 * len(reqs)))
    big = tpm.Context(0)
    ref = {r.rid: r for r in ForceServer(big, source, policy="bh").serve(fresh(reqs), realtime=False)}
    big.close()
    # budget from measurements: the round plan plus 2.2 times the largest
    # resident tree holds that tree's build (its scratch nearly doubles it) but
    # not the five smaller trees (together ~0.9 of it) next to the build
    probe = tpm.Context(0)
    plans = [probe.create_plan(1 << 16, 8)]  # the server's round slot
    plan_bytes = probe.memory()[0]
    tree = probe.build_tree(*source(order[-1]))
    tree_bytes = probe.memory()[0] - plan_bytes
    tree.release()
    for plan in plans:
        plan.close()
    probe.close()
    small = tpm.Context(0, budget_bytes=plan_bytes + int(2.2 * tree_bytes))
    srv = ForceServer(small, source, max_round_ids=1 << 16, max_round_requests=8, policy="bh")
    out = srv.serve(fresh(reqs), realtime=True)
    assert srv.evictions > 0
    for r in out:
        np.testing.assert_array_equal(r.acc, ref[r.rid].acc)
        assert r.latency > 0
    srv.close()
    base = serve_per_request(small, source, fresh(reqs), policy="bh", realtime=True)
    for r in base:
        e = rel(r.acc.astype(np.float64), ref[r.rid].acc.astype(np.float64))
        assert np.percentile(e, 99) < 2e-5
    small.close()


def test_rounds_in_flight_together_give_the_same_results(setup):
    """Two round slots (a request arriving while a round walks starts at once
    on the other stream) against one: the same results, request by request."""
    tpm, torch, cat, source, reqs = setup
    from paper_1909_04667_gb300.serve import ForceServer

    ctx = tpm.Context(0)
    out = {}
    for slots in (1, 2):
        srv = ForceServer(ctx, source, max_round_ids=1 << 18, max_round_requests=4, policy="bh", slots=slots)
        rq = fresh(reqs)
        for r in rq:
            r.arrival = 0.0005 * r.rid  # arrivals faster than the walks: rounds overlap
        out[slots] = {r.rid: r for r in srv.serve(rq, realtime=True)}
        srv.close()
    for rid, r in out[2].items():
        np.testing.assert_array_equal(r.n_int, out[1][rid].n_int)
        e = rel(r.acc.astype(np.float64), out[1][rid].acc.astype(np.float64))
        assert e.max() < 1e-5
    ctx.close()


def test_evicted_system_keeps_its_a_old(setup):
    """An evicted system's |a| comes back with its rebuilt tree: the next
    request on it uses the relative criterion and gets the forces of a plain
    call with that |a| (the same tree, the same walk)."""
    tpm, torch, cat, source, _ = setup
    from paper_1909_04667_gb300.serve import ForceServer, ServeRequest

    sid = max(range(len(cat)), key=lambda i: cat[i].n)
    n = cat[sid].n
    ids = np.arange(n, dtype=np.int32)
    ctx = tpm.Context(0)
    srv = ForceServer(ctx, source, max_round_ids=1 << 18, max_round_requests=8)
    first = srv.serve([ServeRequest(0, sid, ids.copy())], realtime=False)[0]
    assert first.criterion == tpm.CRIT_BH
    assert srv._evict_one() and sid not in srv.resident
    again = srv.serve([ServeRequest(1, sid, ids.copy())], realtime=False)[0]
    assert again.criterion == tpm.CRIT_RELATIVE
    srv.close()
    dev = torch.device("cuda", 0)
    a_old = torch.linalg.vector_norm(torch.from_numpy(first.acc).to(dev), dim=1).contiguous()
    pos, mass, bp = source(sid)
    s = ctx.build_tree(pos, mass, bp)
    a, p, k = s.compute_forces(active_ids=torch.from_numpy(ids).to(dev), a_old=a_old,
                               fp=tpm.ForceParams(crit=tpm.CRIT_RELATIVE, alpha=0.0025))
    np.testing.assert_array_equal(again.acc, a.cpu().numpy())
    np.testing.assert_array_equal(again.n_int, k.cpu().numpy())
    s.release()
    # without the option the rebuilt system starts over with the geometric criterion
    srv = ForceServer(ctx, source, max_round_ids=1 << 18, max_round_requests=8, keep_aold=False)
    srv.serve([ServeRequest(2, sid, ids.copy())], realtime=False)
    assert srv._evict_one()
    assert srv.serve([ServeRequest(3, sid, ids.copy())], realtime=False)[0].criterion == tpm.CRIT_BH
    srv.close()
    ctx.close()
