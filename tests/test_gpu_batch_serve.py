"""Batched and served integration through the C ABI: the persistent kernel and
the serving loop must give each element set the results of its own call (and of
the FP64 oracle), alone and in the mix."""
import threading
import time

import numpy as np
import pytest
import torch

import oracle
from helpers import ORACLE_RULE, TOL, make_inputs, max_errors
from paper_1504_01023_gb300 import api, meshgen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_1504_01023_gb300 import build
    build.build()
    c = api.Context(0)
    yield c
    c.close()


# (type, kind, quad, per-point coefficients, elements, sliver fraction)
MIX = [
    (api.TET, api.POISSON, api.QUAD_TET1, 0, 1, 0.0),
    (api.TET, api.POISSON, api.QUAD_TET4, 1, 5000, 0.0),
    (api.TET, api.GENERIC, api.QUAD_TET4, 0, 12345, 0.05),
    (api.TET, api.GENERIC, api.QUAD_TET1, 1, 33, 0.0),
    (api.TET, api.GENERIC, api.QUAD_TET4, 1, 2000, 0.1),
    (api.PRISM, api.POISSON, api.QUAD_PRISM6, 0, 777, 0.0),
    (api.PRISM, api.POISSON, api.QUAD_PRISM6, 1, 4096, 0.0),
    (api.PRISM, api.GENERIC, api.QUAD_PRISM6, 0, 3001, 0.0),
    (api.PRISM, api.GENERIC, api.QUAD_PRISM6, 1, 6000, 0.0),
    (api.TET, api.GENERIC, api.QUAD_TET4, 0, 129, 0.0),
]


def _set(i, et, kind, quad, cpq, n, frac):
    mesh = (meshgen.tet_cube_mesh(14, seed=40 + i) if et == api.TET else meshgen.prism_slab_mesh(60, seed=40 + i))[:n].copy()
    if frac and et == api.TET:
        meshgen.make_slivers(mesh, frac, seed=90 + i)
    _, c = make_inputs(et, kind, quad, cpq, mesh=mesh, seed=60 + i)
    X = torch.from_numpy(np.ascontiguousarray(mesh)).cuda()
    C = torch.from_numpy(np.ascontiguousarray(c.astype(np.float32).reshape(n, -1))).cuda()
    return mesh, c.astype(np.float32).astype(np.float64), X, C


@pytest.fixture(scope="module")
def mix():
    return [_set(i, *m) for i, m in enumerate(MIX)]


def _items(mix, outs):
    items = []
    for (et, kind, quad, cpq, n, _), (mesh, c, X, C), out in zip(MIX, mix, outs):
        a = api.make_args(et, X, C, kind, quad, api.PER_QPOINT if cpq else api.PER_ELEMENT, api.FP32_MIXED, api.AOS)
        o = api.make_out(*out, api.AOS)
        items.append((et, a, o))
    return items


@pytest.mark.parametrize("autotune", [False, True])
def test_batch_matches_single_calls_and_oracle(ctx, mix, autotune):
    bctx = api.Context(0, autotune=autotune) if autotune else ctx
    outs = [api.alloc_out(et, n, api.FP32_MIXED, api.AOS, "cuda") for (et, kind, quad, cpq, n, _) in MIX]
    items = _items(mix, outs)
    for rep in range(2):                       # first submission captures the graph, second replays it
        for o in outs:
            for t in o:
                t.zero_()
        bctx.batch_submit(items)
        bctx.sync()
        for (et, kind, quad, cpq, n, _), (mesh, c, X, C), out in zip(MIX, mix, outs):
            ref = ctx.integrate(et, X, C, kind, quad, api.PER_QPOINT if cpq else api.PER_ELEMENT, api.FP32_MIXED,
                                api.AOS, api.AOS)
            ctx.sync()
            An, bn, fn = (t.double().cpu().numpy() if t.dtype != torch.uint8 else t.cpu().numpy() for t in out)
            Ar, br, fr = (t.double().cpu().numpy() if t.dtype != torch.uint8 else t.cpu().numpy() for t in ref)
            assert np.array_equal(fn, fr)
            assert oracle.rel_frobenius(An, Ar).max() <= 1e-6
            assert oracle.rel_frobenius(bn, br).max() <= 1e-6
            Ao, bo, _ = oracle.integrate(et, kind, ORACLE_RULE[quad], mesh, c, coef_per_q=bool(cpq), n_threads=8)
            ea, eb = max_errors(An, bn, Ao, bo)
            assert ea <= TOL[api.FP32_MIXED] and eb <= TOL[api.FP32_MIXED], (et, kind, quad, cpq, ea, eb)
    if autotune:
        bctx.close()


@pytest.mark.parametrize("block,tpe,pers", [(64, 2, 1), (128, 2, 0), (32, 1, 1), (256, 1, 0), (64, 1, 0)])
def test_batch_pinned_shapes(mix, block, tpe, pers):
    """Pinned batch shapes, including two threads per prism element and one block
    per tile instead of persistent grids: every set against the oracle, flags as in
    a single call."""
    bctx = api.Context(0)
    bctx.batch_set_shape(block, tpe, pers)
    outs = [api.alloc_out(et, n, api.FP32_MIXED, api.AOS, "cuda") for (et, kind, quad, cpq, n, _) in MIX]
    items = _items(mix, outs)
    bctx.batch_submit(items)
    bctx.batch_submit(items)                    # graph replay
    bctx.sync()
    for (et, kind, quad, cpq, n, _), (mesh, c, X, C), out in zip(MIX, mix, outs):
        An, bn, fn = (t.double().cpu().numpy() if t.dtype != torch.uint8 else t.cpu().numpy() for t in out)
        ref = bctx.integrate(et, X, C, kind, quad, api.PER_QPOINT if cpq else api.PER_ELEMENT, api.FP32_MIXED,
                             api.AOS, api.AOS)
        bctx.sync()
        assert np.array_equal(fn, ref[2].cpu().numpy())
        Ao, bo, _ = oracle.integrate(et, kind, ORACLE_RULE[quad], mesh, c, coef_per_q=bool(cpq), n_threads=8)
        ea, eb = max_errors(An, bn, Ao, bo)
        assert ea <= TOL[api.FP32_MIXED] and eb <= TOL[api.FP32_MIXED], (et, kind, quad, cpq, ea, eb)
    with pytest.raises(api.FeError):
        bctx.batch_set_shape(256, 2)                 # 512 threads
    with pytest.raises(api.FeError):
        bctx.batch_set_shape(48, 1)                  # not a multiple of 32
    bctx.batch_set_shape(None)
    bctx.close()


def test_batch_rejects_unsupported_items(ctx, mix):
    (et, kind, quad, cpq, n, _), (mesh, c, X, C) = MIX[2], mix[2]
    out = api.alloc_out(et, n, api.FP32_MIXED, api.SOA, "cuda")
    a = api.make_args(et, X, C, kind, quad, api.PER_ELEMENT, api.FP32_MIXED, api.AOS)
    o = api.make_out(*out, api.SOA)
    with pytest.raises(api.FeError) as e:
        ctx.batch_submit([(et, a, o)])
    assert e.value.status == -6


def _register(ctx, et, mesh, how):
    if how == "aos-host":
        return ctx.mesh_register(et, torch.from_numpy(np.ascontiguousarray(mesh)), api.AOS)
    if how == "aos-dev":
        return ctx.mesh_register(et, torch.from_numpy(np.ascontiguousarray(mesh)).cuda(), api.AOS)
    if how == "soa-host":
        return ctx.mesh_register(et, torch.from_numpy(meshgen.soa(mesh)), api.SOA)
    return ctx.mesh_register(et, torch.from_numpy(meshgen.soa(mesh)).cuda(), api.SOA)


def _wait(ctx, tk, timeout=30.0):
    t0 = time.time()
    while True:
        r = ctx.serve_poll(tk)
        if r is not None:
            return r
        assert time.time() - t0 < timeout, "request did not finish"
        time.sleep(0.0005)


def test_serve_alone_and_in_the_mix(ctx, mix):
    hows = ["aos-host", "aos-dev", "soa-host", "soa-dev"]
    reqs = []
    for i, ((et, kind, quad, cpq, n, _), (mesh, c, X, C)) in enumerate(zip(MIX, mix)):
        mid = _register(ctx, et, mesh, hows[i % 4])
        reqs.append((mid, et, kind, quad, api.PER_QPOINT if cpq else api.PER_ELEMENT, C, mesh, c))
    # one large set (generic prisms, per-point coefficients) keeps the device busy in the mix
    big_mesh = meshgen.prism_slab_mesh(800, seed=77)                        # 1,280,000 prisms
    _, big_c = make_inputs(api.PRISM, api.GENERIC, api.QUAD_PRISM6, 1, mesh=big_mesh, seed=78)
    big_C = torch.from_numpy(big_c.astype(np.float32).reshape(len(big_mesh), -1)).cuda()
    big_id = _register(ctx, api.PRISM, big_mesh, "aos-host")
    reqs.append((big_id, api.PRISM, api.GENERIC, api.QUAD_PRISM6, api.PER_QPOINT, big_C, None, None))
    # alone: one request at a time
    alone = []
    for mid, et, kind, quad, cm, C, mesh, c in reqs:
        tk = ctx.serve_submit(mid, kind, quad, cm, C)
        r = _wait(ctx, tk)
        assert r.status == 0 and r.t_submit_us <= r.t_launch_us <= r.t_done_us
        A, b, f = ctx.serve_result_tensors(tk, r)
        alone.append((A.double().cpu().numpy(), b.double().cpu().numpy(), f.cpu().numpy()))
        ctx.serve_release(tk)
    # the oracle for each small set
    for (mid, et, kind, quad, cm, C, mesh, c), (An, bn, fn) in zip(reqs[:-1], alone):
        Ao, bo, _ = oracle.integrate(et, kind, ORACLE_RULE[quad], mesh, c, coef_per_q=cm == api.PER_QPOINT, n_threads=8)
        ea, eb = max_errors(An, bn, Ao, bo)
        assert ea <= TOL[api.FP32_MIXED] and eb <= TOL[api.FP32_MIXED]
    # in the mix: the large request six times first (about a millisecond of GPU
    # work), then every small one once from this thread and twice more from two
    # threads while they run
    big = len(reqs) - 1
    tickets = [(big, ctx.serve_submit(*(reqs[big][:1] + reqs[big][2:6]))) for _ in range(6)]
    lock = threading.Lock()

    def client(order):
        for j in order:
            mid, et, kind, quad, cm, C, mesh, c = reqs[j]
            tk = ctx.serve_submit(mid, kind, quad, cm, C)
            with lock:
                tickets.append((j, tk))

    client(list(range(big)))
    idx = list(range(big)) * 2
    th = [threading.Thread(target=client, args=(idx[k::2],)) for k in range(2)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    spans = {}
    for j, tk in tickets:
        r = _wait(ctx, tk)
        assert r.status == 0
        spans[tk] = (j, r.t_launch_us, r.t_done_us)
        A, b, f = ctx.serve_result_tensors(tk, r)
        An, bn, fn = A.double().cpu().numpy(), b.double().cpu().numpy(), f.cpu().numpy()
        assert np.array_equal(fn, alone[j][2])
        assert oracle.rel_frobenius(An, alone[j][0]).max() <= 1e-6
        assert oracle.rel_frobenius(bn, alone[j][1]).max() <= 1e-6
        ctx.serve_release(tk)
    # requests that arrived while the large ones ran were launched before the last
    # of them finished
    bd = max(d for tk, (j, l, d) in spans.items() if j == big)
    overlapped = sum(1 for tk, (j, l, d) in spans.items() if j != big and l < bd)
    assert overlapped > 0
    for mid, *_ in reqs:
        ctx.mesh_release(mid)


def test_serve_fp64_request(ctx, mix):
    (et, kind, quad, cpq, n, _), (mesh, c, X, C) = MIX[7], mix[7]
    mid = _register(ctx, et, mesh, "aos-dev")
    C64 = torch.from_numpy(np.ascontiguousarray(c.reshape(n, -1))).cuda()
    tk = ctx.serve_submit(mid, kind, quad, api.PER_ELEMENT, C64, prec=api.FP64)
    r = _wait(ctx, tk)
    A, b, f = ctx.serve_result_tensors(tk, r)
    Ao, bo, _ = oracle.integrate(et, kind, ORACLE_RULE[quad], mesh, c, n_threads=8)
    ea, eb = max_errors(A.cpu().numpy(), b.cpu().numpy(), Ao, bo)
    assert ea <= TOL[api.FP64] and eb <= TOL[api.FP64]
    ctx.serve_release(tk)
    ctx.mesh_release(mid)


def test_serve_budget(mix):
    (et, kind, quad, cpq, n, _), (mesh, c, X, C) = MIX[2], mix[2]
    mesh_bytes = n * 12 * 8
    out_bytes = 3 * 256 + n * (16 + 4) * 4 + n
    with api.Context(0, hbm_budget=mesh_bytes + out_bytes + 4096) as small:
        mid = small.mesh_register(et, torch.from_numpy(np.ascontiguousarray(mesh)), api.AOS)
        t1 = small.serve_submit(mid, kind, quad, api.PER_ELEMENT, C)
        t2 = small.serve_submit(mid, kind, quad, api.PER_ELEMENT, C)   # waits for t1's release
        r1 = _wait(small, t1)
        time.sleep(0.05)
        assert small.serve_poll(t2) is None                          # not admitted yet
        small.serve_release(t1)
        r2 = _wait(small, t2)
        assert r2.status == 0 and r2.t_launch_us >= r1.t_done_us
        # a request waiting for budget can be withdrawn; one that ran cannot
        t3 = small.serve_submit(mid, kind, quad, api.PER_ELEMENT, C)
        time.sleep(0.05)
        assert small.serve_poll(t3) is None                          # waits for t2's release
        small.serve_cancel(t3)
        with pytest.raises(api.FeError):
            small.serve_poll(t3)
        with pytest.raises(api.FeError):
            small.serve_cancel(t2)
        small.serve_release(t2)
        time.sleep(0.05)
        assert small.serve_wait_any(timeout_us=20000) == []         # t3 never runs
        # a mesh that can never fit
        with pytest.raises(api.FeError) as e:
            small.mesh_register(et, torch.from_numpy(np.ascontiguousarray(meshgen.tet_cube_mesh(30))), api.AOS)
        assert e.value.status == -3
        small.mesh_release(mid)


def test_serve_completion_queue(ctx, mix):
    """fe_serve_wait_any returns every finished request once, in completion order,
    with the results fe_serve_poll reports; a request released before it is
    returned is skipped."""
    ids = []
    for i, ((et, kind, quad, cpq, n, _), (mesh, c, X, C)) in enumerate(zip(MIX, mix)):
        ids.append((_register(ctx, et, mesh, "aos-dev"), kind, quad, api.PER_QPOINT if cpq else api.PER_ELEMENT, C))
    assert ctx.serve_wait_any(timeout_us=0) == []
    submitted = [ctx.serve_submit(*args) for args in ids * 3]
    # one request finished and released through poll before the queue returns it
    skip = submitted[0]
    _wait(ctx, skip)
    ctx.serve_release(skip)
    got = {}
    t0 = time.time()
    while len(got) < len(submitted) - 1:
        for tk, r in ctx.serve_wait_any(timeout_us=20000, max_results=5):
            assert tk not in got and tk != skip
            got[tk] = r
        assert time.time() - t0 < 30, "completion queue stalled"
    assert set(got) == set(submitted[1:])
    done_times = [got[tk].t_done_us for tk in got]
    assert done_times == sorted(done_times)                   # completion order
    for tk, r in got.items():
        p = ctx.serve_poll(tk)
        assert p.status == r.status == 0 and p.A == r.A and p.t_done_us == r.t_done_us
        ctx.serve_release(tk)
    assert ctx.serve_wait_any(timeout_us=1000) == []
    for mid, *_ in ids:
        ctx.mesh_release(mid)


def test_serve_submit_and_release_many(ctx, mix):
    """fe_serve_submit_n queues every request or none; the results equal those of
    single submissions; fe_serve_release_n releases every ticket or none."""
    ids = []
    for i, ((et, kind, quad, cpq, n, _), (mesh, c, X, C)) in enumerate(zip(MIX, mix)):
        ids.append((_register(ctx, et, mesh, "aos-dev"), kind, quad, api.PER_QPOINT if cpq else api.PER_ELEMENT, C))
    # single submissions, for reference
    ref = {}
    for j, args in enumerate(ids):
        tk = ctx.serve_submit(*args)
        r = _wait(ctx, tk)
        A, b, f = ctx.serve_result_tensors(tk, r)
        ref[j] = (A.cpu().numpy().copy(), b.cpu().numpy().copy(), f.cpu().numpy().copy())
        ctx.serve_release(tk)
    # a bad request in the middle: nothing is queued
    bad = list(ids)
    bad.insert(3, (10 ** 9,) + ids[0][1:])                     # unknown mesh id
    with pytest.raises(api.FeError) as e:
        ctx.serve_submit_many(bad)
    assert e.value.status == -1
    assert ctx.serve_wait_any(timeout_us=20000) == []
    # all of them at once, twice
    tks = ctx.serve_submit_many(ids + ids)
    assert len(set(tks)) == 2 * len(ids)
    rs = [_wait(ctx, tk) for tk in tks]
    launches = {r.t_launch_us for r in rs}
    assert len(launches) < len(tks)                          # they shared launches
    for k, (tk, r) in enumerate(zip(tks, rs)):
        assert r.status == 0
        A, b, f = ctx.serve_result_tensors(tk, r)
        An, bn, fn = ref[k % len(ids)]
        assert np.array_equal(f.cpu().numpy(), fn)
        assert oracle.rel_frobenius(A.double().cpu().numpy(), An.astype(np.float64)).max() <= 1e-6
        assert oracle.rel_frobenius(b.double().cpu().numpy(), bn.astype(np.float64)).max() <= 1e-6
    # a repeated or unknown ticket releases none
    with pytest.raises(api.FeError):
        ctx.serve_release_many([tks[0], tks[0]])
    with pytest.raises(api.FeError):
        ctx.serve_release_many([tks[1], 10 ** 12])
    assert ctx.serve_poll(tks[0]).status == 0 and ctx.serve_poll(tks[1]).status == 0
    ctx.serve_release_many(tks)
    for tk in tks:
        with pytest.raises(api.FeError):
            ctx.serve_poll(tk)
    ctx.serve_release_many([])
    assert ctx.serve_submit_many([]) == []
    # the completion queue skips what was released before it was returned
    while ctx.serve_wait_any(timeout_us=0):
        pass
    for mid, *_ in ids:
        ctx.mesh_release(mid)


def test_serve_concurrent_clients_stress(ctx, mix):
    """Four client threads submit (one by one and in groups), cancel and release
    while a fifth drains the completion queue: every request that was not
    cancelled completes exactly once, with the results of its single call."""
    import random
    ids, refs = [], []
    for i, ((et, kind, quad, cpq, n, _), (mesh, c, X, C)) in enumerate(zip(MIX, mix)):
        cm = api.PER_QPOINT if cpq else api.PER_ELEMENT
        ids.append((_register(ctx, et, mesh, "aos-dev"), kind, quad, cm, C))
        A, b, f = ctx.integrate(et, X, C, kind, quad, cm, api.FP32_MIXED, api.AOS, api.AOS)
        ctx.sync()
        refs.append((A.double().cpu().numpy(), b.double().cpu().numpy(), f.cpu().numpy()))
    lock = threading.Lock()
    owner, cancelled, done = {}, set(), {}
    errors = []
    stop = threading.Event()

    def client(seed):
        rng = random.Random(seed)
        try:
            for _ in range(60):
                k = rng.randint(1, 4)
                js = [rng.randrange(len(ids)) for _ in range(k)]
                tks = ctx.serve_submit_many([ids[j] for j in js]) if k > 1 else [ctx.serve_submit(*ids[js[0]])]
                with lock:
                    owner.update(zip(tks, js))
                if rng.random() < 0.3:
                    tk = rng.choice(tks)
                    try:
                        ctx.serve_cancel(tk)
                        with lock:
                            cancelled.add(tk)
                    except api.FeError:
                        pass                      # already launched: it completes normally
        except Exception as e:                    # noqa: BLE001
            errors.append(e)

    def owner_of(tk):
        # a completion can arrive before its client has recorded the ticket
        t0 = time.time()
        while time.time() - t0 < 10:
            with lock:
                if tk in owner:
                    return owner[tk]
            time.sleep(0.0002)
        return None

    def collector():
        deadline = time.time() + 120
        while time.time() < deadline:
            got = ctx.serve_wait_any(timeout_us=20000, max_results=32)
            for tk, r in got:
                j = owner_of(tk)
                with lock:
                    if j is None or tk in done or tk in cancelled:
                        errors.append(("unexpected completion", tk))
                        continue
                    done[tk] = r
                A, b, f = ctx.serve_result_tensors(tk, r)
                An, bn, fn = refs[j]
                if not (r.status == 0 and np.array_equal(f.cpu().numpy(), fn) and
                        oracle.rel_frobenius(A.double().cpu().numpy(), An).max() <= 1e-6 and
                        oracle.rel_frobenius(b.double().cpu().numpy(), bn).max() <= 1e-6):
                    errors.append(("mismatch", tk, j))
            if got:
                ctx.serve_release_many([tk for tk, _ in got])
            with lock:
                finished = stop.is_set() and len(done) + len(cancelled) == len(owner)
            if finished:
                return

    def collector_guarded():
        try:
            collector()
        except Exception as e:                    # noqa: BLE001
            errors.append(("collector", repr(e)))

    col = threading.Thread(target=collector_guarded, daemon=True)
    col.start()
    clients = [threading.Thread(target=client, args=(s,)) for s in range(4)]
    for t in clients:
        t.start()
    for t in clients:
        t.join()
    stop.set()
    col.join(timeout=150)
    assert not col.is_alive(), "completion queue stalled"
    assert not errors, errors[:3]
    assert set(done) | cancelled == set(owner) and not (set(done) & cancelled)
    for mid, *_ in ids:
        ctx.mesh_release(mid)
