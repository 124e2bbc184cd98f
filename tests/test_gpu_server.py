"""The continuous-batching server (tabnet_server_*) on the GPU.

The paper's GPU functions keep the model resident and answer batches of
records with predictions and attribution masks (Sec. III-B); here many
requests of three resident models are served at once.  A request's result
must be the same alone and in a mix (rows are independent), and admission by
device memory must hold requests back rather than fail them.
"""
import math

import numpy as np
import pytest

from oracle import tabnet_oracle as O
from paper_2510_19689_b300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

NAMES = ["c1", "c2", "c3"]


@pytest.fixture(scope="module")
def models():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_19689_b300 import tabnet
    params = [synth.make_params(synth.SPECS[n], 70 + i, bn_affine="random") for i, n in enumerate(NAMES)]
    ms = [tabnet.Model(synth.to_blob(p), "bf16x3") for p in params]
    yield tabnet, params, ms
    for m in ms:
        m.close()


def _req(name, rows, seed):
    return synth.make_rows(name, rows, seed=seed)


def test_same_result_alone_and_in_a_mix(models):
    tabnet, params, ms = models
    # one batch in flight at a time: requests that arrive meanwhile queue up
    # and leave together in the next batch
    srv = tabnet.Server(ms, device_bytes=256 << 20, max_inflight_batches=1)
    targets = [(i, *_req(n, r, 100 + i)) for i, (n, r) in enumerate(zip(NAMES, [37, 300, 129]))]
    alone = []
    for i, xn, xc in targets:
        t = srv.submit(i, xn, xc)
        srv.wait(t)
        alone.append(srv.result(t))
        srv.release(t)
    # the same requests again, each in the middle of a burst of other requests
    rng = np.random.default_rng(5)
    burst = []
    for k in range(300):
        i = int(rng.integers(3))
        burst.append((i, *_req(NAMES[i], int(rng.integers(1, 200)), 1000 + k)))
    tickets, mine = [], {}
    for k, (i, xn, xc) in enumerate(burst):
        tickets.append(srv.submit(i, xn, xc))
        if k in (100, 150, 200):
            j = (100, 150, 200).index(k)
            mine[j] = srv.submit(targets[j][0], targets[j][1], targets[j][2])
    for j, t in mine.items():
        srv.wait(t)
        for a, b in zip(alone[j], srv.result(t)):
            np.testing.assert_array_equal(a, b)
        srv.release(t)
    for t in tickets:
        srv.wait(t)
        srv.release(t)
    st = srv.stats()
    assert st["rejected"] == 0 and st["completed"] == st["submitted"]
    assert st["batches"] < st["submitted"]  # requests were batched together
    srv.close()
    # and against the oracle (split-bf16 bar)
    for (i, xn, xc), (lg, mk, ag) in zip(targets, alone):
        rl, rm, ra = O.forward(params[i], xn, xc)
        assert np.abs(lg - rl).max() <= 2e-2
        assert np.abs(mk - rm).sum(axis=(1, 2)).max() <= 2e-2
        assert np.abs(ag - ra).sum(axis=1).max() <= 2e-2


def test_admission_waits_for_memory(models):
    """Rings sized for a few hundred rows of the 100-input model: requests
    submitted faster than they complete find its input ring full, queue
    unstaged and are copied in by the engine later, in order -- and still
    give the same bits as a direct forward of their rows."""
    tabnet, params, ms = models
    srv = tabnet.Server(ms, device_bytes=8 << 20, max_batch_rows=512)
    tickets, reqs = [], []
    for k in range(60):
        i = k % 3
        xn, xc = _req(NAMES[i], 200, 2000 + k)
        reqs.append((i, xn, xc))
        tickets.append(srv.submit(i, xn, xc))
    results = []
    for t in tickets:
        srv.wait(t, 60.0)
        results.append(srv.result(t))
        srv.release(t)
    st = srv.stats()
    assert st["completed"] == 60 and st["rejected"] == 0
    assert st["engine_staged"] > 0  # the full-ring path ran
    for (i, xn, xc), got in zip(reqs, results):
        ref = ms[i].run(torch.from_numpy(xn).cuda(), torch.from_numpy(xc).cuda())
        for a, b in zip(got, ref):
            np.testing.assert_array_equal(a, b.cpu().numpy())
    # a request larger than its model's whole ring is rejected, not hung
    xn, xc = _req("c3", 4000, 3000)
    srv.submit(2, xn, xc)
    for _ in range(200):
        if srv.stats()["rejected"] == 1:
            break
        import time
        time.sleep(0.01)
    assert srv.stats()["rejected"] == 1
    srv.close()


@pytest.mark.parametrize("threads", [1, 4])
def test_poisson_replay(models, threads):
    tabnet, params, ms = models
    srv = tabnet.Server(ms, device_bytes=512 << 20)
    rng = np.random.default_rng(9)
    pools = [_req(n, 512, 4000 + i) for i, n in enumerate(NAMES)]
    n_req, rate = 3000, 20000.0
    t = np.cumsum(rng.exponential(1.0 / rate, n_req))
    sizes = np.minimum(512, np.floor(np.exp(rng.uniform(0, math.log(513), n_req)))).astype(int)
    reqs = []
    for k in range(n_req):
        i = int(rng.integers(3))
        xn, xc = pools[i]
        reqs.append((i, xn[:sizes[k]], xc[:sizes[k]], float(t[k])))
    srv.reset_stats()
    srv.replay(reqs, threads=threads, warmup=n_req // 10)
    st = srv.stats()
    assert st["completed"] == n_req and st["rejected"] == 0
    assert st["rows_completed"] == int(sizes.sum())
    assert 0 < st["p50_ms"] <= st["p99_ms"] <= st["max_ms"]
    # every request's wait for its launch is part of its latency
    assert 0 <= st["p50_queue_ms"] <= st["p50_ms"] and st["p99_queue_ms"] <= st["p99_ms"]
    assert 0.0 <= st["engine_busy"] <= 1.0
    srv.close()


def test_same_result_under_the_default_policy(models):
    """Default server shape (8 streams and 32 in-flight batches per model,
    adaptive batching under load) with a float32-accurate model resident
    beside the split-bf16 ones: requests answered inside a dense burst equal
    the same requests answered alone, bit for bit."""
    tabnet, params, ms = models
    p6 = synth.make_params(synth.SPECS["c2"], 79, bn_affine="random")
    m6 = tabnet.Model(synth.to_blob(p6), "bf16x6")
    resident = ms + [m6]
    names = NAMES + ["c2"]
    srv = tabnet.Server(resident, device_bytes=512 << 20)
    targets = [(i, *_req(names[i], r, 200 + i)) for i, r in zip(range(4), [5, 77, 33, 260])]
    alone = []
    for i, xn, xc in targets:
        t = srv.submit(i, xn, xc)
        srv.wait(t)
        alone.append(srv.result(t))
        srv.release(t)
    rng = np.random.default_rng(6)
    tickets, mine = [], {}
    for k in range(2000):
        i = int(rng.integers(4))
        tickets.append(srv.submit(i, *_req(names[i], int(rng.integers(1, 120)), 3000 + k)))
        if k % 500 == 250:
            j = k // 500
            mine[j] = srv.submit(targets[j][0], targets[j][1], targets[j][2])
    for j, t in mine.items():
        srv.wait(t)
        for a, b in zip(alone[j], srv.result(t)):
            np.testing.assert_array_equal(a, b)
        srv.release(t)
    for t in tickets:
        srv.wait(t)
        srv.release(t)
    st = srv.stats()
    assert st["rejected"] == 0 and st["completed"] == st["submitted"]
    srv.close()
    m6.close()
    # the float32-accurate model's answer against the oracle at the float32 bar
    i, xn, xc = targets[3]
    lg = alone[3][0]
    rl = O.forward(p6, xn, xc)[0]
    assert (np.abs(lg - rl) / np.maximum(np.abs(rl), 1)).max() <= 1e-5


def test_mask_transfer_modes_are_exact(models):
    """Step masks travel to the host compact (per row-step the nonzero
    columns and their values) where that saves bytes; a batch with a row-step
    over the slot count travels densely.  Compact (default slots), compact
    overflowing into the dense fallback (one slot) and always dense must give
    the same bits, equal to a direct forward of the same rows, and the
    compact form must decode to those masks."""
    tabnet, params, ms = models
    reqs = [(i, *_req(n, r, 300 + 7 * i + r)) for i, n in enumerate(NAMES) for r in (1, 64, 257)]
    direct = []
    for i, xn, xc in reqs:
        lg, mk, ag = ms[i].run(torch.from_numpy(xn).cuda(), torch.from_numpy(xc).cuda())
        direct.append((lg.cpu().numpy(), mk.cpu().numpy(), ag.cpu().numpy()))
    for slots in (0, 1, -1):
        srv = tabnet.Server(ms, device_bytes=256 << 20, mask_slots=slots)
        tickets = [srv.submit(i, xn, xc) for i, xn, xc in reqs]
        for t, (i, xn, xc), ref in zip(tickets, reqs, direct):
            srv.wait(t)
            got = srv.result(t)
            for a, b in zip(got, ref):
                np.testing.assert_array_equal(a, b)
            comp = srv.result_compact(t)
            if slots == 0 and NAMES[i] in ("c2", "c3"):
                assert comp is not None  # compact on the wide models, no overflow at these slot counts
            if slots == -1 or (slots == 0 and NAMES[i] == "c1"):
                assert comp is None      # dense by request, or the narrow model (no saving)
            if comp is not None:
                cnt, col, val = comp
                mk = got[1]
                np.testing.assert_array_equal(cnt, (mk != 0).sum(axis=2))
                dec = np.zeros_like(mk)
                for (r, s) in np.ndindex(cnt.shape):
                    dec[r, s, col[r, s, :cnt[r, s]]] = val[r, s, :cnt[r, s]]
                np.testing.assert_array_equal(dec, mk)
            srv.release(t)
        srv.close()
