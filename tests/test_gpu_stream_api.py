"""The ticketed stream API through the C ABI: semr_open / semr_submit /
semr_query / semr_fetch / semr_close.

These calls are the library's hand-over point: a producer submits a snapshot
that lives in device memory and goes on, and fetches the reduced payload and
the error report when it is ready -- the asynchronous in-situ approach of
arXiv 2407.20731, Sec. III-A, where the application waits only for the
hand-over.  Checked here: results through the stream equal the FP64 oracle;
a ticket reports SEMR_EAGAIN until its work is done; the memory budget
refuses a ticket that does not fit; a too-small payload buffer keeps the
ticket; a ticket whose codes outgrow the first payload estimate is re-run at
its exact size and still equals the oracle; unknown tickets are refused;
closing with tickets outstanding frees them.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle
import paper_2407_20731_b300 as semr
from parity import compare_payloads, make_case

pytestmark = pytest.mark.gpu


def _oracle_check(fields, jac, tau, payload, reps, elem):
    f_np, j_np = fields.cpu().numpy(), jac.cpu().numpy()
    o = oracle.reduce(f_np, j_np, tau, fragile_cap=100000)
    compare_payloads(payload, o.payload, o.fragile)
    F = f_np.shape[0]
    umax = np.abs(f_np).reshape(F, -1).max(axis=1)
    np.testing.assert_allclose(elem[:, :, 1], o.elem_report[:, :, 1], rtol=1e-12, atol=0)
    assert np.all(np.abs(elem[:, :, 2] - o.elem_report[:, :, 2]) <= 1e-12 * umax[:, None])
    d = 1e-12 * umax[:, None]
    J = j_np[None, :]
    bound = 2 * d * np.sqrt(8 * J * o.elem_report[:, :, 0]) + 8 * J * d * d + 1e-12 * o.elem_report[:, :, 0]
    assert np.all(np.abs(elem[:, :, 0] - o.elem_report[:, :, 0]) <= bound)
    for f in range(F):
        assert reps[f].umax == o.field_report[f, 6]
        assert reps[f].kept == int(o.field_report[f, 7])
        np.testing.assert_allclose(reps[f].sum_energy, o.field_report[f, 5], rtol=1e-12)
        np.testing.assert_allclose(reps[f].l2_rel, o.field_report[f, 1], rtol=1e-9)


def _submit(h, fields, jac, lx, tau, precision=semr.SEMR_FP64, cumulative=False):
    fs = semr.make_fieldset([fields[i] for i in range(fields.shape[0])], tau, precision, cumulative=cumulative)
    rc, t = semr.semr_submit(h, fs, semr.make_mesh(lx, jac))
    return rc, t


def _fetch(h, t, fields, wait=True):
    F, E = fields.shape[0], fields.shape[1]
    lx = round((fields.shape[2]) ** (1 / 3))
    sz = semr.semr_sizes_for(lx, E, F, 1e-3)
    buf = np.zeros(int(sz.payload_worst), dtype=np.uint8)
    elem = np.zeros((F, E, 3))
    rc, nb, reps = semr.semr_fetch(h, t, wait, buf, F, elem)
    return rc, buf[:nb], reps, elem


def test_three_tickets_equal_the_oracle():
    """Three snapshots (lx 8 and 6, one to three fields) submitted at once,
    polled, then fetched out of order: every payload, field report and
    element report equals the oracle's."""
    cases = [make_case(700, 8, 2, seed=71), make_case(333, 6, 1, seed=72), make_case(129, 8, 3, seed=73)]
    lxs = [8, 6, 8]
    h = semr.semr_open(0, 0, 0)
    try:
        tickets = []
        for (f, j), lx in zip(cases, lxs):
            rc, t = _submit(h, f, j, lx, 1e-3)
            assert rc == semr.SEMR_OK
            tickets.append(t)
        assert len(set(tickets)) == 3
        for t in tickets:
            for _ in range(200000):
                rc = semr.semr_query(h, t)
                if rc != semr.SEMR_EAGAIN:
                    break
            assert rc == semr.SEMR_OK
        for k in (2, 0, 1):
            f, j = cases[k]
            rc, payload, reps, elem = _fetch(h, tickets[k], f)
            assert rc == semr.SEMR_OK
            _oracle_check(f, j, 1e-3, payload, reps, elem)
            # a fetched ticket is gone
            assert semr.semr_query(h, tickets[k]) == semr.SEMR_EINVAL
            assert _fetch(h, tickets[k], f)[0] == semr.SEMR_EINVAL
    finally:
        semr.semr_close(h)


@pytest.mark.parametrize("lx", [6, 8, 10])
def test_cumulative_ticket_equals_the_oracle(lx):
    """A cumulative-truncation ticket (FP64 mode) next to a threshold one on
    the same stream: the fetched payload equals the oracle's cumulative
    variant outside its fragile list and the single launch byte for byte,
    and its field reports match the oracle."""
    f, j = make_case(900, lx, 2, seed=74 + lx)
    g, k = make_case(500, lx, 1, seed=75 + lx)
    h = semr.semr_open(0, 0, 0)
    try:
        rc, t_cum = _submit(h, f, j, lx, 1e-3, cumulative=True)
        assert rc == semr.SEMR_OK
        rc, t_thr = _submit(h, g, k, lx, 1e-3)
        assert rc == semr.SEMR_OK
        rc, payload, reps, elem = _fetch(h, t_cum, f)
        assert rc == semr.SEMR_OK
        alone = semr.reduce([f[i] for i in range(2)], j, lx, 1e-3, precision=semr.SEMR_FP64, cumulative=True)
        assert np.array_equal(payload, alone.payload)
        o = oracle.reduce(f.cpu().numpy(), j.cpu().numpy(), 1e-3, fragile_cap=100000, cumulative=True)
        compare_payloads(payload, o.payload, o.fragile)
        for fi in range(2):
            assert reps[fi].umax == o.field_report[fi, 6]
            assert reps[fi].kept == int(o.field_report[fi, 7])
            np.testing.assert_allclose(reps[fi].sum_energy, o.field_report[fi, 5], rtol=1e-12)
            np.testing.assert_allclose(reps[fi].l2_rel, o.field_report[fi, 1], rtol=1e-9)
        rc, payload2, _, _ = _fetch(h, t_thr, g)
        assert rc == semr.SEMR_OK
        assert np.array_equal(payload2, semr.reduce([g[0]], k, lx, 1e-3, precision=semr.SEMR_FP64).payload)
    finally:
        semr.semr_close(h)


def test_eagain_until_complete():
    """A ticket queued behind a long device-side delay on the caller's stream
    answers SEMR_EAGAIN to semr_query and to a non-waiting semr_fetch; a
    waiting fetch then returns the results."""
    f, j = make_case(2000, 8, 2, seed=74)
    torch.cuda.synchronize()  # the inputs are complete before the other stream reads them
    s = torch.cuda.Stream()
    h = semr.semr_open(0, s.cuda_stream, 0)
    try:
        with torch.cuda.stream(s):
            torch.cuda._sleep(int(4e8))  # about 0.2 s of GPU time ahead of the reduction
        rc, t = _submit(h, f, j, 8, 1e-3)
        assert rc == semr.SEMR_OK
        assert semr.semr_query(h, t) == semr.SEMR_EAGAIN
        assert _fetch(h, t, f, wait=False)[0] == semr.SEMR_EAGAIN
        assert semr.semr_query(h, t) == semr.SEMR_EAGAIN  # the non-waiting fetch kept the ticket
        rc, payload, reps, elem = _fetch(h, t, f, wait=True)
        assert rc == semr.SEMR_OK
        _oracle_check(f, j, 1e-3, payload, reps, elem)
    finally:
        semr.semr_close(h)


def _ticket_bytes(lx, E, F, tau, fill=1.0 / 32):
    """Device bytes of a fresh stream's first ticket: the payload estimate
    (1/16 of all modes, plus 4096 codes), scratch, summary, report
    (the layout semr_submit documents, with its alignment slack)."""
    sz = semr.semr_sizes_for(lx, E, F, tau)
    modes = F * E * lx ** 3
    cap = min(int(sz.payload_worst), int(sz.code_base) + int(sz.code_width) * int(min(1.0, 2 * fill) * modes + 4096))
    a = lambda b: (b + 255) // 256 * 256  # noqa: E731
    return a(a(cap) + int(sz.scratch_bytes) + ctypes.sizeof(semr.semr_summary) + 512 + int(sz.elem_report_bytes))


def test_budget_refuses_what_does_not_fit():
    f, j = make_case(1000, 8, 2, seed=75)
    one = _ticket_bytes(8, 1000, 2, 1e-3)
    h = semr.semr_open(0, 0, int(one * 1.5))  # room for one ticket, not two
    try:
        rc1, t1 = _submit(h, f, j, 8, 1e-3)
        assert rc1 == semr.SEMR_OK
        rc2, _ = _submit(h, f, j, 8, 1e-3)
        assert rc2 == semr.SEMR_EBUDGET
        rc, payload, reps, elem = _fetch(h, t1, f)
        assert rc == semr.SEMR_OK
        _oracle_check(f, j, 1e-3, payload, reps, elem)
        rc3, t3 = _submit(h, f, j, 8, 1e-3)  # fits again once the first is fetched
        assert rc3 == semr.SEMR_OK
        assert _fetch(h, t3, f)[0] == semr.SEMR_OK
    finally:
        semr.semr_close(h)
    h = semr.semr_open(0, 0, 4096)  # smaller than any ticket
    try:
        assert _submit(h, f, j, 8, 1e-3)[0] == semr.SEMR_EBUDGET
    finally:
        semr.semr_close(h)


def test_small_buffer_keeps_the_ticket():
    f, j = make_case(500, 8, 1, seed=76)
    h = semr.semr_open(0, 0, 0)
    try:
        rc, t = _submit(h, f, j, 8, 1e-3)
        assert rc == semr.SEMR_OK
        small = np.zeros(64, dtype=np.uint8)
        rc, nb, reps = semr.semr_fetch(h, t, True, small, 1)
        assert rc == semr.SEMR_ENOSPACE and nb > 64
        assert semr.semr_query(h, t) == semr.SEMR_OK  # still there
        rc, payload, reps, elem = _fetch(h, t, f)
        assert rc == semr.SEMR_OK and payload.size == nb
        _oracle_check(f, j, 1e-3, payload, reps, elem)
    finally:
        semr.semr_close(h)


def test_codes_beyond_the_estimate_rerun_exactly():
    """White-noise elements keep about half their modes, about three times
    the first ticket's payload estimate: the ticket is re-run at the exact size
    its first run reports, and the results equal the oracle and a direct
    semr_reduce_async; the next ticket of the stream is sized from this fill
    and runs once."""
    E = 400
    f, j = make_case(E, 8, 1, seed=77)
    g = torch.Generator().manual_seed(77)
    f[0] = torch.randn(E, 512, dtype=torch.float64, generator=g).cuda()
    direct = semr.reduce([f[0]], j, 8, 1e-3)
    kept = direct.summary.code_total
    assert kept > (E * 512) // 16 + 4096  # beyond the first estimate
    h = semr.semr_open(0, 0, 0)
    try:
        for _ in range(2):
            rc, t = _submit(h, f, j, 8, 1e-3)
            assert rc == semr.SEMR_OK
            rc, payload, reps, elem = _fetch(h, t, f)
            assert rc == semr.SEMR_OK
            assert payload.size == direct.payload.size and np.array_equal(payload, direct.payload)
            _oracle_check(f, j, 1e-3, payload, reps, elem)
    finally:
        semr.semr_close(h)


@pytest.mark.parametrize("flagged", ["subnormal", "nan"])
def test_rerun_with_input_flags(flagged):
    """A ticket whose codes outgrow the first payload estimate and whose input
    also raises an input flag -- an element of subnormal values only
    (SEMR_STATUS_TINY, informational) or one holding a NaN
    (SEMR_STATUS_NONFINITE) -- is still re-run at the exact size: the fetch
    delivers the complete payload, equal to a direct semr_reduce_async, with
    SEMR_OK or SEMR_ENONFINITE respectively."""
    E = 400
    g = torch.Generator().manual_seed(79)
    f = torch.randn(1, E, 512, dtype=torch.float64, generator=g)
    if flagged == "subnormal":
        f[0, 17] = torch.randn(512, dtype=torch.float64, generator=g) * 1e-310
    else:
        f[0, 17, 100] = float("nan")
    f = f.cuda().contiguous()
    j = (0.5 + 1.5 * torch.rand(E, dtype=torch.float64, generator=g)).cuda().contiguous()
    direct = semr.reduce([f[0]], j, 8, 1e-3)
    flag = semr.SEMR_STATUS_TINY if flagged == "subnormal" else semr.SEMR_STATUS_NONFINITE
    assert direct.summary.status == flag
    assert direct.summary.code_total > (E * 512) // 16 + 4096  # beyond the first estimate
    h = semr.semr_open(0, 0, 0)
    try:
        rc, t = _submit(h, f, j, 8, 1e-3)
        assert rc == semr.SEMR_OK
        rc, payload, reps, elem = _fetch(h, t, f)
        assert rc == (semr.SEMR_OK if flagged == "subnormal" else semr.SEMR_ENONFINITE)
        assert np.array_equal(payload, direct.payload)
        assert np.array_equal(elem, direct.elem_report, equal_nan=True)
    finally:
        semr.semr_close(h)


def test_bad_tickets_and_arguments():
    f, j = make_case(64, 8, 1, seed=78)
    h = semr.semr_open(0, 0, 0)
    try:
        assert semr.semr_query(h, 12345) == semr.SEMR_EINVAL
        assert _fetch(h, 12345, f)[0] == semr.SEMR_EINVAL
        assert _submit(h, f, j, 8, -1.0)[0] == semr.SEMR_EINVAL
        assert _submit(h, f, j, 8, 1e-20)[0] == semr.SEMR_EINVAL  # codes would not fit int32
        assert _submit(h, f, j, 13, 1e-3)[0] == semr.SEMR_EINVAL
    finally:
        semr.semr_close(h)


def test_close_with_tickets_outstanding():
    f, j = make_case(3000, 8, 2, seed=79)
    h = semr.semr_open(0, 0, 0)
    for _ in range(3):
        assert _submit(h, f, j, 8, 1e-3)[0] == semr.SEMR_OK
    semr.semr_close(h)  # waits for the work, frees every ticket
    torch.cuda.synchronize()
    h = semr.semr_open(0, 0, 0)  # the device is still usable
    try:
        rc, t = _submit(h, f, j, 8, 1e-3)
        assert rc == semr.SEMR_OK
        assert _fetch(h, t, f)[0] == semr.SEMR_OK
    finally:
        semr.semr_close(h)


def test_concurrent_submit_query_fetch():
    """Four producer threads share one stream handle, each submitting, polling
    and fetching its own tickets while the others do the same (the calls are
    documented thread-safe with respect to each other): every result equals
    the same reduction through semr_reduce_async, byte for byte."""
    import threading
    cases = [make_case(300 + 150 * i, 8 if i % 2 == 0 else 6, 1 + i % 3, seed=200 + i) for i in range(8)]
    lxs = [8 if i % 2 == 0 else 6 for i in range(8)]
    direct = [semr.reduce([f[k] for k in range(f.shape[0])], j, lx, 1e-3).payload for (f, j), lx in zip(cases, lxs)]
    torch.cuda.synchronize()
    h = semr.semr_open(0, 0, 0)
    errors = []

    def producer(idx):
        try:
            for _ in range(3):
                for i in idx:
                    f, j = cases[i]
                    rc, t = _submit(h, f, j, lxs[i], 1e-3)
                    assert rc == semr.SEMR_OK
                    while semr.semr_query(h, t) == semr.SEMR_EAGAIN:
                        pass
                    rc, payload, reps, elem = _fetch(h, t, f)
                    assert rc == semr.SEMR_OK
                    assert np.array_equal(payload, direct[i]), i
        except Exception as e:  # noqa: BLE001 -- reported by the main thread
            errors.append(e)

    threads = [threading.Thread(target=producer, args=([k, k + 4],)) for k in range(4)]
    try:
        for t in threads:
            t.start()
        for t in threads:
            t.join()
    finally:
        semr.semr_close(h)
    assert not errors, errors
