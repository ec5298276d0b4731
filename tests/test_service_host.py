"""Host logic of the streaming service, run in dry-run mode (no CUDA call):
admission, ring accounting, guaranteed vs unguaranteed readers, batching of
pending gulps, integration boundaries, sequence gaps, flush, output-buffer
back-pressure, host-side fault injection."""
import numpy as np
import pytest

from paper_1708_00720_b300 import service as sv
from paper_1708_00720_b300 import xengine as xe

MiB = 1 << 20


# scratch of the time-sliced leftover units of a plan on a 148-SM B300:
# one slot per CTA pair, one 128 x 128 int2 tile per CTA
SPLIT_WS = 74 * 2 * 128 * 128 * 8


def dev_bytes(N, C, T, R):
    nbl = N * (N + 1) // 2
    return R * T * C * N + 2 * C * nbl * 8 + SPLIT_WS + MiB


def mk(manual=True, cap=1 << 34):
    return sv.Service(mem_cap_bytes=cap, dryrun=True, manual=manual)


def put(s, sid, seq):
    v = s.reserve(s_id := sid)
    assert v is not None
    v[:] = seq % 251
    s.commit(s_id, seq)


def test_admission_against_the_cap():
    need, small = dev_bytes(64, 32, 128, 4), dev_bytes(16, 1, 16, 1)
    s = mk(cap=2 * need + small + (need - small) // 2)
    a = s.add_stream(64, 32, 128, ring_gulps=4)
    b = s.add_stream(64, 32, 128, ring_gulps=4)
    assert s.stats(a)["device_bytes"] == need and s.stats(b)["device_bytes"] == need
    with pytest.raises(xe.XEngineError) as e:
        s.add_stream(64, 32, 128, ring_gulps=4)
    assert e.value.status == xe.XE_ERR_NOMEM and "admission" in str(e.value)
    s.add_stream(16, 1, 16, ring_gulps=1)   # a small one still fits


def test_stream_argument_checks():
    s = mk()
    with pytest.raises(xe.XEngineError) as e:
        s.add_stream(20, 1, 16)
    assert e.value.status == xe.XE_ERR_ALIGNMENT
    with pytest.raises(xe.XEngineError) as e:
        s.add_stream(16, 4, 1 << 20, integrate_gulps=32)        # 2^25 samples > int32 bound
    assert e.value.status == xe.XE_ERR_ACCUM_BOUND
    with pytest.raises(xe.XEngineError) as e:
        s.add_stream(16, 4, 1 << 16, integrate_gulps=4, out="cf32")   # 2^18 > exact-float bound
    assert e.value.status == xe.XE_ERR_ACCUM_BOUND
    with pytest.raises(xe.XEngineError):
        s.add_stream(16, 4, 16, ring_gulps=0)
    with pytest.raises(xe.XEngineError):
        sv.Service(mem_cap_bytes=0, dryrun=True)               # a dry run needs an explicit cap


def test_unguaranteed_ring_skips_when_full_then_batches():
    s = mk()
    a = s.add_stream(16, 16, 4, ring_gulps=4, integrate_gulps=100, guaranteed=False)
    for q in range(4):
        put(s, a, q)
    st = s.stats(a)
    assert (st["inflight"], st["pending"], st["launches"]) == (2, 2, 2)
    assert s.reserve(a) is None                     # full ring: the gulp is skipped
    assert s.stats(a)["skipped_full"] == 1
    s.dryrun_complete(a)                            # the two launches finish
    st = s.stats(a)
    assert st["launches"] == 3 and st["max_batch"] == 2 and st["pending"] == 0
    assert st["gulps_correlated"] == 4


def test_guaranteed_ring_reports_busy_without_skipping():
    s = mk()
    a = s.add_stream(16, 16, 4, ring_gulps=2, integrate_gulps=100, guaranteed=True)
    put(s, a, 0)
    put(s, a, 1)
    assert s.reserve(a, timeout_ms=10) is None
    assert s.stats(a)["skipped_full"] == 0
    s.dryrun_complete(a)
    assert s.reserve(a) is not None


def test_batches_stop_at_the_ring_wrap_and_at_integration_boundaries():
    s = mk()
    a = s.add_stream(16, 16, 4, ring_gulps=6, integrate_gulps=4, guaranteed=False)
    for q in range(6):                              # slots 0..5; launches: {0}, {1}; pending 2..5
        put(s, a, q)
    s.dryrun_complete(a)
    st = s.stats(a)
    # pending seqs 2, 3 (integration 0) go together; 4, 5 (integration 1) wait for the emit
    assert st["max_batch"] == 2 and st["integrations"] == 1
    s.dryrun_complete(a)
    st = s.stats(a)
    assert st["gulps_correlated"] == 6 and st["max_batch"] == 2
    for q in range(6, 9):                           # slots 0, 1, 2 after the wrap
        put(s, a, q)
    s.dryrun_complete(a)
    s.dryrun_complete(a)
    assert s.stats(a)["gulps_correlated"] == 9


def test_integration_boundaries_gaps_and_flush():
    s = mk(manual=False)
    a = s.add_stream(16, 16, 4, ring_gulps=8, integrate_gulps=4, guaranteed=True)
    for q in (0, 1, 2, 3):
        put(s, a, q)
    r = s.poll(a)
    assert (r["index"], r["first_seq"], r["gulps"], r["skipped"], r["samples"]) == (0, 0, 4, 0, 16)
    assert r["vis"].shape == (16, 16 * 17 // 2, 2) and not r["vis"].any()
    s.release(a, 0)
    for q in (4, 5, 7):                             # seq 6 never arrives
        put(s, a, q)
    assert s.poll(a) is None                        # integration 1 still open
    put(s, a, 9)                                    # the writer moved on: integration 1 closes
    r = s.poll(a)
    assert (r["index"], r["gulps"], r["skipped"], r["samples"]) == (1, 3, 1, 12)
    s.release(a, 1)
    s.flush(a)                                      # integration 2 holds only seq 9
    r = s.poll(a)
    assert (r["index"], r["first_seq"], r["gulps"], r["skipped"]) == (2, 8, 1, 3)
    s.release(a, 2)
    assert s.stats(a)["integrations"] == 3


def test_flush_with_nothing_open_does_not_cut_the_next_integration():
    """A flush after an integration has already closed applies to nothing:
    the next integration's first gulp must not be emitted alone (a stale
    flush once closed it after one gulp and emitted the rest a second time
    under the same index)."""
    s = mk(manual=False)
    a = s.add_stream(16, 16, 4, ring_gulps=8, integrate_gulps=4, guaranteed=True)
    for q in range(4):
        put(s, a, q)
    r = s.poll(a)
    assert (r["index"], r["gulps"]) == (0, 4)
    s.release(a, 0)
    s.flush(a)                                      # integration 0 is already out
    put(s, a, 4)
    assert s.poll(a) is None                        # integration 1 stays open
    for q in (5, 6, 7):
        put(s, a, q)
    r = s.poll(a)
    assert (r["index"], r["first_seq"], r["gulps"], r["skipped"]) == (1, 4, 4, 0)
    s.release(a, 1)
    assert s.stats(a)["integrations"] == 2


def test_sequence_numbers_must_increase():
    s = mk(manual=False)
    a = s.add_stream(16, 16, 4, ring_gulps=4, integrate_gulps=4)
    put(s, a, 5)
    s.reserve(a)
    with pytest.raises(xe.XEngineError) as e:
        s.commit(a, 5)
    assert e.value.status == xe.XE_ERR_INVALID_ARG
    s.reserve(a)
    s.commit(a, 6)                                  # the slot was handed back; the stream goes on


def test_output_buffers_apply_back_pressure():
    s = mk(manual=False)
    a = s.add_stream(16, 16, 4, ring_gulps=3, integrate_gulps=1, guaranteed=True)
    put(s, a, 0)
    put(s, a, 1)                                    # two integrations hold both output buffers
    put(s, a, 2)                                    # correlated; its emit must wait
    put(s, a, 3)                                    # 3, 4, 5 cannot be correlated before that emit
    put(s, a, 4)
    put(s, a, 5)
    st = s.stats(a)
    assert st["integrations"] == 2 and st["pending"] == 3
    assert s.reserve(a, timeout_ms=5) is None       # ring full behind the blocked emit
    r0 = s.poll(a)
    s.release(a, r0["index"])
    st = s.stats(a)
    assert st["integrations"] == 3 and st["pending"] == 2   # 2 emitted; 3 correlated, its emit waits again
    assert s.reserve(a) is not None


def test_fault_injection_isolates_the_stream():
    s = mk(manual=False)
    a = s.add_stream(16, 16, 4, ring_gulps=4, integrate_gulps=2)
    b = s.add_stream(16, 16, 4, ring_gulps=4, integrate_gulps=2)
    s.inject(a, sv.XE_FAULT_LAUNCH)
    put(s, a, 0)
    assert s.stats(a)["state"] == xe.XE_ERR_CUDA
    with pytest.raises(xe.XEngineError) as e:
        s.reserve(a)
    assert e.value.status == xe.XE_ERR_CUDA
    for q in range(2):
        put(s, b, q)
    r = s.poll(b)
    assert r["gulps"] == 2 and s.stats(b)["state"] == xe.XE_OK


def test_dropped_gulp_is_reported_as_skipped():
    s = mk(manual=False)
    a = s.add_stream(16, 16, 4, ring_gulps=4, integrate_gulps=3)
    put(s, a, 0)
    s.inject(a, sv.XE_FAULT_DROP_GULP)
    put(s, a, 1)                                    # lost in transit
    put(s, a, 2)
    s.flush(a)
    r = s.poll(a)
    assert (r["gulps"], r["skipped"], r["samples"]) == (2, 1, 8)
    assert s.stats(a)["dropped"] == 1


def test_streams_are_independent():
    s = mk(manual=False)
    ids = [s.add_stream(16 * (k + 1), 16, 4, ring_gulps=4, integrate_gulps=2) for k in range(3)]
    for q in range(4):
        for i in ids:
            put(s, i, q)
    for k, i in enumerate(ids):
        for idx in range(2):
            r = s.poll(i)
            assert r["index"] == idx and r["vis"].shape[1] == (16 * (k + 1)) * (16 * (k + 1) + 1) // 2
            s.release(i, idx)


def test_service_needs_a_gpu_outside_dry_run(gpu_available):
    if gpu_available:
        pytest.skip("a GPU is present")
    with pytest.raises(xe.XEngineError):
        sv.Service()


def test_ready_gulps_of_several_streams_share_a_launch():
    # the GPU takes two launches in flight; further ready gulps wait, and when
    # the GPU frees up the e4m3 streams' runs go in ONE launch, the int32
    # stream's on its own (manual dry run: work completes on request)
    s = mk()
    a = s.add_stream(64, 8, 128, ring_gulps=8, integrate_gulps=1)
    b = s.add_stream(128, 4, 256, ring_gulps=8, integrate_gulps=1)
    c = s.add_stream(64, 8, 128, ring_gulps=8, integrate_gulps=1, operand="int32")
    put(s, a, 0)
    put(s, b, 0)                              # two launches in flight: the GPU is busy
    put(s, c, 0)
    put(s, a, 1)
    put(s, b, 1)
    assert [s.stats(x)["inflight"] for x in (a, b, c)] == [1, 1, 0]
    assert [s.stats(x)["pending"] for x in (a, b, c)] == [1, 1, 1]
    s.dryrun_complete(-1)
    sa, sb, sc = s.stats(a), s.stats(b), s.stats(c)
    assert (sa["shared_launches"], sb["shared_launches"], sc["shared_launches"]) == (1, 1, 0)
    assert (sa["launches"], sb["launches"], sc["launches"]) == (2, 2, 1)
    assert sa["pending"] == sb["pending"] == sc["pending"] == 0
    for sid, n in ((a, 2), (b, 2), (c, 1)):
        for idx in range(n):
            s.dryrun_complete(sid)
            r = s.poll(sid, timeout_ms=1000)
            assert (r["index"], r["gulps"], r["skipped"]) == (idx, 1, 0)
            s.release(sid, idx)
    s.close()


def test_no_batch_flag_keeps_launches_to_one_stream():
    s = sv.Service(mem_cap_bytes=1 << 34, dryrun=True, manual=True, batch=False)
    a = s.add_stream(64, 8, 128, ring_gulps=8, integrate_gulps=1)
    b = s.add_stream(64, 8, 128, ring_gulps=8, integrate_gulps=1)
    put(s, a, 0)
    put(s, b, 0)
    put(s, a, 1)
    put(s, b, 1)
    s.dryrun_complete(-1)
    assert s.stats(a)["shared_launches"] == 0 and s.stats(b)["shared_launches"] == 0
    assert s.stats(a)["launches"] == 2 and s.stats(b)["launches"] == 2
    s.close()
