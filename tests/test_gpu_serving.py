"""The serving form: requests submitted while others run are admitted into
device slots as slots and memory free up, and their kernels overlap on the
GPU.  Each result must be the same alone and in the mix (byte-identical:
the kernels are deterministic and each request has its own buffers)."""
import threading

import numpy as np
import pytest

import oracle
import paper_2407_20731_b300 as semr
from parity import compare_payloads, make_case

pytestmark = pytest.mark.gpu

SHAPES = [(4096, 8, 3, 1e-6), (700, 6, 1, 1e-5), (2500, 10, 2, 1e-6), (64, 8, 4, 1e-4), (3000, 6, 2, 1e-6),
          (1500, 8, 1, 1e-5), (900, 10, 3, 1e-6), (5000, 8, 2, 1e-7)]


def _requests():
    reqs = []
    for i, (ne, lx, nf, tau) in enumerate(SHAPES):
        f, j = make_case(ne, lx, nf, seed=80 + i)
        reqs.append(([f[k] for k in range(nf)], j, lx, tau))
    return reqs


def _alone(req, precision):
    fields, jac, lx, tau = req
    return semr.reduce(fields, jac, lx, tau, precision=precision).payload


@pytest.mark.parametrize("precision", [semr.SEMR_FP32, semr.SEMR_FP64])
def test_each_result_same_alone_and_in_the_mix(precision):
    reqs = _requests()
    alone = [_alone(r, precision) for r in reqs]
    srv = semr.Server(slots=4)
    ids = []
    lock = threading.Lock()

    def producer(sub):
        for i in sub:
            rid = srv.submit(*reqs[i], precision=precision)
            with lock:
                ids.append((rid, i))

    threads = [threading.Thread(target=producer, args=(list(range(len(reqs)))[k::3],)) for k in range(3)]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    for rid, i in ids:
        rc, info = srv.wait(rid)
        assert rc == semr.SEMR_OK
        assert info.t_submit <= info.t_admit <= info.t_done
        buf = np.zeros(int(info.summary.payload_bytes), dtype=np.uint8)
        rc, n = srv.release(rid, buf)
        assert rc == semr.SEMR_OK and n == buf.size
        assert np.array_equal(buf, alone[i])
    st = srv.stats()
    assert st["completed"] == len(reqs) and st["held_bytes"] == 0
    srv.close()


def test_budget_queues_and_rejects():
    reqs = _requests()
    # what the server reserves per request (payload estimate or exact re-run size, scratch, reports)
    probe = semr.Server(slots=1)
    sizes = []
    for r in reqs:
        rid = probe.submit(*r)
        rc, info = probe.wait(rid)
        assert rc == semr.SEMR_OK
        sizes.append(int(info.device_bytes))
        probe.release(rid)
    probe.close()
    budget = int(max(sizes) * 1.3)  # only about one request fits at a time
    srv = semr.Server(slots=4, mem_budget_bytes=budget)
    ids = [srv.submit(*r) for r in reqs]
    slots_seen = set()
    for rid in ids:
        rc, info = srv.wait(rid)
        assert rc == semr.SEMR_OK
        slots_seen.add(info.slot)
        srv.release(rid)
    assert srv.stats()["held_bytes"] == 0
    srv.close()
    tiny = semr.Server(slots=1, mem_budget_bytes=1024)
    with pytest.raises(semr.SemrError) as e:
        tiny.submit(*reqs[0])
    assert e.value.code == semr.SEMR_EBUDGET
    tiny.close()


def test_codes_beyond_the_estimate_rerun_exactly():
    """A white-noise snapshot keeps about half its modes, far beyond the
    server's first payload estimate (1/16 of the modes plus 4096 codes): its
    request is re-run on its slot at the exact size the first run reports,
    and the result equals the same reduction alone; requests after it are
    sized from that fill and run once."""
    import torch
    E = 400
    g = torch.Generator().manual_seed(91)
    f = torch.randn(1, E, 512, dtype=torch.float64, generator=g).cuda().contiguous()
    j = (0.5 + 1.5 * torch.rand(E, dtype=torch.float64, generator=g)).cuda().contiguous()
    req = ([f[0]], j, 8, 1e-3)
    alone = _alone(req, semr.SEMR_FP64)
    sz = semr.semr_sizes_for(8, E, 1, 1e-3)
    kept = (alone.size - int(sz.code_base)) // 2
    assert kept > (E * 512) // 16 + 4096  # beyond the first estimate
    srv = semr.Server(slots=2)
    for _ in range(2):
        rid = srv.submit(*req, precision=semr.SEMR_FP64)
        rc, info = srv.wait(rid)
        assert rc == semr.SEMR_OK and info.summary.status == 0
        assert info.device_bytes >= info.summary.payload_bytes
        buf = np.zeros(int(info.summary.payload_bytes), dtype=np.uint8)
        rc, _ = srv.release(rid, buf)
        assert rc == semr.SEMR_OK and np.array_equal(buf, alone)
    assert srv.stats()["held_bytes"] == 0
    srv.close()


@pytest.mark.parametrize("flagged", ["subnormal", "nan"])
def test_rerun_with_input_flags(flagged):
    """A request beyond the first payload estimate whose input also raises an
    input flag (an element of subnormal values only: SEMR_STATUS_TINY,
    informational; a NaN: SEMR_STATUS_NONFINITE) is still re-run at the exact
    size: the released payload is complete and equals the reduction alone."""
    import torch
    E = 400
    g = torch.Generator().manual_seed(92)
    f = torch.randn(1, E, 512, dtype=torch.float64, generator=g)
    if flagged == "subnormal":
        f[0, 33] = torch.randn(512, dtype=torch.float64, generator=g) * 1e-310
    else:
        f[0, 33, 7] = float("nan")
    f = f.cuda().contiguous()
    j = (0.5 + 1.5 * torch.rand(E, dtype=torch.float64, generator=g)).cuda().contiguous()
    req = ([f[0]], j, 8, 1e-3)
    alone = semr.reduce(*req, precision=semr.SEMR_FP64)
    flag = semr.SEMR_STATUS_TINY if flagged == "subnormal" else semr.SEMR_STATUS_NONFINITE
    assert alone.summary.status == flag
    srv = semr.Server(slots=2)
    rid = srv.submit(*req, precision=semr.SEMR_FP64)
    rc, info = srv.wait(rid)
    assert rc == (semr.SEMR_OK if flagged == "subnormal" else semr.SEMR_ENONFINITE)
    assert info.summary.status == flag
    buf = np.zeros(int(info.summary.payload_bytes), dtype=np.uint8)
    rc, _ = srv.release(rid, buf)
    assert rc == semr.SEMR_OK and np.array_equal(buf, alone.payload)
    srv.close()


def test_served_results_equal_the_oracle():
    """FP64 mode through the server, all eight requests in flight together on
    four slots: every served payload equals the FP64 oracle's outside its
    fragile list, and every field report matches it."""
    reqs = _requests()
    srv = semr.Server(slots=4)
    ids = [srv.submit(*r, precision=semr.SEMR_FP64) for r in reqs]
    for rid, (fields, jac, lx, tau) in zip(ids, reqs):
        rc, info = srv.wait(rid)
        assert rc == semr.SEMR_OK
        buf = np.zeros(int(info.summary.payload_bytes), dtype=np.uint8)
        rc, _ = srv.release(rid, buf)
        assert rc == semr.SEMR_OK
        f_np = np.stack([f.cpu().numpy() for f in fields])
        o = oracle.reduce(f_np, jac.cpu().numpy(), tau, fragile_cap=100000)
        compare_payloads(buf, o.payload, o.fragile)
        for f in range(len(fields)):
            assert info.summary.field[f].umax == o.field_report[f, 6]
            np.testing.assert_allclose(info.summary.field[f].sum_energy, o.field_report[f, 5], rtol=1e-12)
            # the 1e-12 max|u| reconstruction tolerance allows ~1e-8 relative on L2_rel at tau = 1e-7
            np.testing.assert_allclose(info.summary.field[f].l2_rel, o.field_report[f, 1], rtol=1e-6)
    srv.close()


def test_cumulative_requests_in_the_mix():
    """Cumulative-energy truncation through the server, mixed with threshold
    requests on the same slots (lx 6, 8 and 10, FP64 mode): every served
    payload equals its single launch byte for byte, and the cumulative ones
    equal the oracle's cumulative variant outside its fragile list.  The
    cumulative budget keeps more codes than the threshold, so these requests
    also exercise the payload estimate and its exact re-run."""
    reqs = _requests()[:6]
    cum = [True, False, True, False, True, True]
    alone = [semr.reduce(f, j, lx, tau, precision=semr.SEMR_FP64, cumulative=c).payload
             for (f, j, lx, tau), c in zip(reqs, cum)]
    srv = semr.Server(slots=3)
    ids = [srv.submit(*r, precision=semr.SEMR_FP64, cumulative=c) for r, c in zip(reqs, cum)]
    for k, rid in enumerate(ids):
        rc, info = srv.wait(rid)
        assert rc == semr.SEMR_OK
        buf = np.zeros(int(info.summary.payload_bytes), dtype=np.uint8)
        rc, _ = srv.release(rid, buf)
        assert rc == semr.SEMR_OK
        assert np.array_equal(buf, alone[k])
        if cum[k]:
            fields, jac, lx, tau = reqs[k]
            f_np = np.stack([f.cpu().numpy() for f in fields])
            o = oracle.reduce(f_np, jac.cpu().numpy(), tau, fragile_cap=100000, cumulative=True)
            compare_payloads(buf, o.payload, o.fragile)
    assert srv.stats()["held_bytes"] == 0
    srv.close()

