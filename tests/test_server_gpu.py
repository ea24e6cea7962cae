"""Request server: resident compressed matrices, admission by a device-memory
budget, continuous batching.  Each result must be the same alone (single-op
entry points) and in the mix: bit for bit for compress / add / sub / scale,
within the dot and product tolerances otherwise.  Failures (unknown handle,
budget, released operand) are produced on the host; nothing here faults or
hangs a GPU."""
import threading
import time

import numpy as np
import pytest
import torch

import oracle as O
import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    from paper_2202_13007_gb300 import _build, blaz

    _build.build()
    blaz.lib()
    return blaz


def same_cmat(x, y):
    for u, v in zip(x.to_host(), y.to_host()):
        u, v = np.asarray(u), np.asarray(v)
        if u.dtype == np.float64:
            assert np.array_equal(u.view(np.uint64), v.view(np.uint64))
        else:
            assert np.array_equal(u, v)


def test_results_alone_and_in_the_mix(B):
    srv = B.Server(budget_bytes=8 << 30, streams=3, max_wait_us=200)
    rng = np.random.default_rng(0)
    shapes = [(64, 128), (256, 256), (8, 8), (520, 136), (1024, 1024)]
    mats = {sh: [W.bump_field(sh[1], 100 + i + sh[0], rows=sh[0]) for i in range(2)] for sh in shapes}
    handles = {}
    for sh, (X, Y) in mats.items():
        ta, tb = srv.submit("compress", A=X), srv.submit("compress", A=Y)
        handles[sh] = (srv.wait(ta)["handle"], srv.wait(tb)["handle"])
    # a mixed stream from two submitting threads
    jobs, lock = [], threading.Lock()

    def producer(seed):
        r = np.random.default_rng(seed)
        for _ in range(60):
            sh = shapes[r.integers(len(shapes))]
            ha, hb = handles[sh]
            kind = ["add", "sub", "scale", "dot", "decompress", "matmul"][r.integers(6)]
            if kind in ("add", "sub"):
                t = srv.submit(kind, a=ha, b=hb)
                item = (kind, sh, t, None, None)
            elif kind == "scale":
                cst = float(r.uniform(-3, 3))
                t = srv.submit("scale", a=ha, c=cst)
                item = (kind, sh, t, cst, None)
            elif kind == "dot":
                out = np.full(1, np.nan)
                t = srv.submit("dot", a=ha, b=hb, out=out)
                item = (kind, sh, t, out, None)
            elif kind == "decompress":
                out = np.full(sh, np.nan)
                t = srv.submit("decompress", a=ha, out=out)
                item = (kind, sh, t, out, None)
            else:
                Bm = r.standard_normal((sh[1], int(r.integers(1, 70))))
                out = np.full((sh[0], Bm.shape[1]), np.nan)
                t = srv.submit("matmul", a=ha, B=Bm, out=out)
                item = (kind, sh, t, out, Bm)
            with lock:
                jobs.append(item)
            time.sleep(float(r.exponential(2e-4)))

    th = [threading.Thread(target=producer, args=(s,)) for s in (1, 2)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    alone = {sh: (B.compress(torch.from_numpy(X).cuda()), B.compress(torch.from_numpy(Y).cuda()))
             for sh, (X, Y) in mats.items()}
    for sh, (ha, hb) in handles.items():   # resident matrices == compress alone, and == oracle
        same_cmat(srv.cmat(ha), alone[sh][0])
        oc = O.compress(mats[sh][0])
        assert np.array_equal(srv.cmat(ha).code.cpu().numpy(), oc.code)
    for kind, sh, t, extra, Bm in jobs:
        res = srv.wait(t)
        assert res["status"] == 0, res
        ga, gb = alone[sh]
        if kind == "add":
            same_cmat(srv.cmat(res["handle"]), B.add(ga, gb))
        elif kind == "sub":
            same_cmat(srv.cmat(res["handle"]), B.sub(ga, gb))
        elif kind == "scale":
            same_cmat(srv.cmat(res["handle"]), B.scale(ga, extra))
        elif kind == "dot":
            want = float(B.dot(ga, gb).item())
            absum = float((B.decompress(ga).abs() * B.decompress(gb).abs()).sum())
            assert abs(extra[0] - want) <= 2e-12 * absum and extra[0] == res["value"]
        elif kind == "decompress":
            want = B.decompress(ga).cpu().numpy()
            assert np.all(np.abs(extra - want) <= 1e-12 * (np.abs(want).max() + 1))
        else:
            Bt = torch.from_numpy(Bm).cuda()
            want = B.matmul(ga, Bt, mode="fp64").cpu().numpy()
            bound = np.abs(B.decompress(ga).cpu().numpy()) @ np.abs(Bm)
            assert np.all(np.abs(extra - want) <= 2e-12 * bound + 1e-300)
    st = srv.stats()
    assert st["completed"] >= len(jobs) + 2 * len(shapes)
    assert st["launches"] < st["completed"]          # requests were batched together
    assert st["p99_us"] >= st["p50_us"] > 0
    srv.destroy()


def test_admission_by_memory_budget(B):
    budget = 3 << 20                                   # 3 MiB
    srv = B.Server(budget_bytes=budget, streams=2)
    X = W.bump_field(256, 7)                           # 512 KiB input, ~23 KiB compressed
    tickets = [srv.submit("compress", A=X) for _ in range(24)]
    res = [srv.wait(t) for t in tickets]
    assert all(r["status"] == 0 for r in res)
    st = srv.stats()
    assert st["peak_bytes"] <= budget
    big = np.zeros((1024, 1024))                       # 8 MiB input can never fit
    with pytest.raises(B.BlazError) as e:
        srv.submit("compress", A=big)
    assert e.value.status == -8
    # releasing frees the resident bytes
    for r in res:
        srv.wait(srv.submit("release", a=r["handle"]))
    assert srv.stats()["resident_bytes"] == 0
    srv.destroy()


def test_release_and_invalid_handles(B):
    srv = B.Server(budget_bytes=1 << 30)
    X = W.bump_field(64, 3)
    h = srv.wait(srv.submit("compress", A=X))["handle"]
    out = np.zeros(1)
    t_dot = srv.submit("dot", a=h, b=h, out=out)       # submitted before the release
    t_rel = srv.submit("release", a=h)
    assert srv.wait(t_dot)["status"] == 0              # the earlier request still completes
    assert srv.wait(t_rel)["status"] == 0
    with pytest.raises(B.BlazError) as e:
        srv.submit("scale", a=h, c=2.0)                # released handle
    assert e.value.status == -9
    with pytest.raises(B.BlazError):
        srv.submit("dot", a=12345, b=12345, out=out)   # unknown handle
    with pytest.raises(B.BlazError) as e:
        srv.submit("compress", A=np.zeros((12, 8)))    # not a multiple of 8
    assert e.value.status == -1
    srv.destroy()


def test_continuous_batching_versus_one_request_per_launch(B):
    reqs = W.poisson_requests(rate=4000, duration_s=0.25, seed=13, lo=64, hi=512)
    shapes = sorted({(d["rows"], d["cols"]) for d in reqs})[:24]
    base = {sh: W.bump_field(sh[1], 5, rows=sh[0]) for sh in shapes}

    def run(max_batch):
        srv = B.Server(budget_bytes=4 << 30, streams=4 if max_batch != 1 else 1, max_batch=max_batch)
        hs = {sh: srv.wait(srv.submit("compress", A=base[sh]))["handle"] for sh in shapes}
        outs, ts = [], []
        t0 = time.perf_counter()
        for i, d in enumerate(reqs):
            sh = shapes[i % len(shapes)]
            delay = d["t"] - (time.perf_counter() - t0)
            if delay > 0:
                time.sleep(delay)
            if d["op"] == "compress":
                ts.append(srv.submit("compress", A=base[sh]))
            elif d["op"] == "dot":
                o = np.zeros(1)
                outs.append(o)
                ts.append(srv.submit("dot", a=hs[sh], b=hs[sh], out=o))
            elif d["op"] == "matmul":
                Bm = np.ones((sh[1], 16))
                o = np.zeros((sh[0], 16))
                outs.append((o, Bm))
                ts.append(srv.submit("matmul", a=hs[sh], B=Bm, out=o))
            else:
                ts.append(srv.submit("scale" if d["op"] == "scale" else "add", a=hs[sh], b=hs[sh], c=2.0))
        for t in ts:
            assert srv.wait(t)["status"] == 0
        st = srv.stats()
        srv.destroy()
        return st

    batched = run(0)
    single = run(1)
    assert single["launches"] == single["completed"]
    assert batched["launches"] < batched["completed"]
    print(f"\nbatched: p50 {batched['p50_us']:.0f} us p99 {batched['p99_us']:.0f} us "
          f"{batched['throughput_rps']:.0f} req/s mean batch {batched['mean_batch']:.1f}; "
          f"one per launch: p50 {single['p50_us']:.0f} us p99 {single['p99_us']:.0f} us "
          f"{single['throughput_rps']:.0f} req/s")


def test_pinned_requests_and_split_bf16_products(B):
    """Page-locked host buffers are used in place; split-bf16 products in the
    server equal the single-op split-bf16 product."""
    srv = B.Server(budget_bytes=2 << 30, streams=2, matmul_mode="split_bf16")
    src = torch.empty((256, 512), dtype=torch.float64, pin_memory=True)
    src.copy_(torch.from_numpy(W.bump_field(512, 9, rows=256)))
    X = src.numpy()
    h = srv.wait(srv.submit("compress", A=X[:128, 8:264], pinned=True))["handle"]   # strided view
    alone = B.compress(torch.from_numpy(np.ascontiguousarray(X[:128, 8:264])).cuda())
    same_cmat(srv.cmat(h), alone)
    Bm = torch.empty((256, 40), dtype=torch.float64, pin_memory=True)
    Bm.copy_(torch.randn(256, 40, dtype=torch.float64))
    out = torch.full((128, 40), np.nan, dtype=torch.float64, pin_memory=True)
    dot = torch.full((1,), np.nan, dtype=torch.float64, pin_memory=True)
    t1 = srv.submit("matmul", a=h, B=Bm.numpy(), out=out.numpy(), pinned=True)
    t2 = srv.submit("dot", a=h, b=h, out=dot.numpy(), pinned=True)
    assert srv.wait(t1)["status"] == 0
    r2 = srv.wait(t2)
    assert r2["status"] == 0 and r2["value"] == float(dot[0])
    want = B.matmul(alone, Bm.cuda(), mode="split_bf16").cpu()
    bound = B.decompress(alone).abs().cpu() @ Bm.abs()
    assert torch.all((out - want).abs() <= 1e-6 * bound + 1e-300)
    assert abs(float(dot[0]) - float(B.dot(alone, alone).item())) <= 1e-12 * float(
        (B.decompress(alone) ** 2).sum())
    srv.destroy()
