"""Streaming service on the GPU: every emitted integration is compared bit
for bit with the oracle's correlation of exactly the gulps that entered it
(gaps and drops included); a failed stream leaves the others correct;
back-pressure; and the bounded device-side wait used for failure detection."""
import time

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sv():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1708_00720_b300 import service
    return service


def gulps_for(N, C, T, n, seed):
    x = synth.voltages(N, C, T * n, seed=seed, random_phase=True, tone_chan=0)
    return [np.ascontiguousarray(x[k * T:(k + 1) * T]) for k in range(n)]


def expect(gulps):
    return oracle.correlate(np.concatenate(gulps, axis=0))


STREAMS = [(32, 16, 64), (64, 8, 128), (144, 4, 96)]   # (N, C, T)


@pytest.mark.parametrize("operand", ["fp8", "int32"])
def test_three_streams_bit_exact(sv, operand):
    s = sv.Service()
    G = 3
    ids, data = [], []
    for k, (N, C, T) in enumerate(STREAMS):
        ids.append(s.add_stream(N, C, T, ring_gulps=4, integrate_gulps=G, operand=operand))
        data.append(gulps_for(N, C, T, 2 * G, seed=50 + k))
    for q in range(2 * G):                          # interleaved writers
        for sid, gl in zip(ids, data):
            assert s.submit(sid, gl[q], q, timeout_ms=5000)
    for sid, gl in zip(ids, data):
        for idx in range(2):
            r = s.poll(sid, timeout_ms=10000)
            assert r is not None and r["status"] == 0
            assert (r["index"], r["gulps"], r["skipped"]) == (idx, G, 0)
            assert r["latency_ms"] > 0
            np.testing.assert_array_equal(r["vis"], expect(gl[idx * G:(idx + 1) * G]))
            s.release(sid, idx)
        st = s.stats(sid)
        assert st["state"] == 0 and st["gulps_correlated"] == 2 * G and st["launches"] <= 2 * G
    s.close()


def test_gap_drop_and_flush_on_gpu(sv):
    N, C, T, G = 64, 8, 64, 4
    s = sv.Service()
    a = s.add_stream(N, C, T, ring_gulps=4, integrate_gulps=G)
    gl = gulps_for(N, C, T, 8, seed=61)
    s.submit(a, gl[0], 0)
    s.submit(a, gl[1], 1)
    s.submit(a, gl[3], 3)                           # seq 2 never arrives
    s.inject(a, sv.XE_FAULT_DROP_GULP)
    s.submit(a, gl[4], 4)                           # dropped in transit; closes integration 0
    s.submit(a, gl[5], 5)
    r = s.poll(a, timeout_ms=10000)
    assert (r["index"], r["gulps"], r["skipped"], r["samples"]) == (0, 3, 1, 3 * T)
    np.testing.assert_array_equal(r["vis"], expect([gl[0], gl[1], gl[3]]))
    s.release(a, 0)
    s.flush(a)
    r = s.poll(a, timeout_ms=10000)
    assert (r["index"], r["gulps"], r["skipped"]) == (1, 1, 3)
    np.testing.assert_array_equal(r["vis"], expect([gl[5]]))
    s.release(a, 1)
    assert s.stats(a)["dropped"] == 1
    s.close()


def test_failed_stream_leaves_others_correct(sv):
    s = sv.Service()
    a = s.add_stream(32, 16, 64, ring_gulps=4, integrate_gulps=2)
    b = s.add_stream(48, 8, 64, ring_gulps=4, integrate_gulps=2)
    ga, gb = gulps_for(32, 16, 64, 2, 70), gulps_for(48, 8, 64, 2, 71)
    s.inject(a, sv.XE_FAULT_LAUNCH)
    s.submit(a, ga[0], 0)
    time.sleep(0.05)
    assert s.stats(a)["state"] != 0
    with pytest.raises(Exception):
        s.submit(a, ga[1], 1)
    for q in range(2):
        s.submit(b, gb[q], q)
    r = s.poll(b, timeout_ms=10000)
    np.testing.assert_array_equal(r["vis"], expect(gb))
    s.release(b, 0)
    s.close()


def test_guaranteed_stream_back_pressure(sv):
    N, C, T = 32, 16, 64
    s = sv.Service()
    a = s.add_stream(N, C, T, ring_gulps=2, integrate_gulps=1, guaranteed=True)
    gl = gulps_for(N, C, T, 6, 72)
    q = 0
    # nobody releases the two output buffers: the third emit waits, then the ring fills
    while q < 6 and s.submit(a, gl[q], q, timeout_ms=300):
        q += 1
    assert q < 6
    assert s.stats(a)["skipped_full"] == 0
    done = []
    for idx in range(2):
        r = s.poll(a, timeout_ms=5000)
        np.testing.assert_array_equal(r["vis"], expect([gl[r["index"]]]))
        done.append(r["index"])
    for idx in done:
        s.release(a, idx)
    assert s.submit(a, gl[q], q, timeout_ms=5000)     # the writer proceeds again
    s.close()


def test_bounded_device_wait_reports_timeout_and_context_survives(sv):
    import torch
    from paper_1708_00720_b300 import xengine as xe
    flag = torch.zeros(1, dtype=torch.int32, device="cuda")
    status = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    t0 = time.perf_counter()
    sv.xe_wait_flag(flag, 1, 200_000_000, status)    # nothing ever sets the flag
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    assert status.item() == 1 and 0.15 < dt < 5.0
    flag.fill_(7)
    sv.xe_wait_flag(flag, 7, 200_000_000, status)
    torch.cuda.synchronize()
    assert status.item() == 0
    x = synth.voltages(16, 16, 32, seed=3)
    eng = xe.XEngine(16, 16, 32)                     # the context still works
    eng.correlate(torch.from_numpy(x).cuda())
    v = eng.integrate()
    torch.cuda.synchronize()
    np.testing.assert_array_equal(v.cpu().numpy(), oracle.correlate(x))
    eng.close()


def test_serving_workload_shapes_bit_exact(sv):
    """The serving workload's three streams (256 inputs x 64 channels, 512 x
    128, 1024 x 256; gulps of 1024 samples, rings of 8, integrations of 8
    gulps) through the service at once.  Each stream's first integration is
    compared with the oracle on every baseline: all channels of the 256-input
    stream, 16 channels of the 512-input one and 8 of the 1024-input one (the
    oracle's cost grows with N^2)."""
    shapes = [(256, 64, 1024), (512, 128, 1024), (1024, 256, 1024)]
    checked = [np.arange(64), np.arange(0, 128, 8), np.arange(0, 256, 32)]
    G = 8
    s = sv.Service()
    ids, data = [], []
    for k, (N, C, T) in enumerate(shapes):
        ids.append(s.add_stream(N, C, T, ring_gulps=8, integrate_gulps=G, guaranteed=True))
        data.append(gulps_for(N, C, T, G, seed=80 + k))
    for q in range(G):                              # interleaved writers
        for sid, gl in zip(ids, data):
            assert s.submit(sid, gl[q], q, timeout_ms=20000)
    for sid, gl, chans in zip(ids, data, checked):
        r = s.poll(sid, timeout_ms=60000)
        assert r is not None and r["status"] == 0
        assert (r["index"], r["gulps"], r["skipped"]) == (0, G, 0)
        x = np.concatenate(gl, axis=0)
        want = oracle.correlate(np.ascontiguousarray(x[:, chans, :]))
        np.testing.assert_array_equal(r["vis"][chans], want)
        s.release(sid, 0)
        assert s.stats(sid)["state"] == 0
    print("\nlaunches shared between streams:", [s.stats(sid)["shared_launches"] for sid in ids],
          "of", [s.stats(sid)["launches"] for sid in ids])
    s.close()


def test_small_stream_is_not_held_behind_a_large_copy(sv):
    """Host-link copies of one direction run in submission order, so the
    service issues them in pieces with the streams taking turns: a small
    stream's integration, emitted just after a large stream's 1 GB
    visibility copy has started, must come back long before that copy ends
    (whole copies kept it waiting for all of it).  Both stay bit-exact."""
    big, small = (1024, 256, 64), (64, 8, 64)
    s = sv.Service()
    a = s.add_stream(*big, ring_gulps=2, integrate_gulps=1, guaranteed=True)
    b = s.add_stream(*small, ring_gulps=2, integrate_gulps=1, guaranteed=True)
    ga = gulps_for(*big, 2, seed=90)
    gb = gulps_for(*small, 2, seed=91)
    lat = {a: [], b: []}
    for q in range(2):
        assert s.submit(a, ga[q], q, timeout_ms=20000)
        time.sleep(0.002)                           # the large copy is under way
        assert s.submit(b, gb[q], q, timeout_ms=20000)
        for sid, gl, chans in ((b, gb, np.arange(8)), (a, ga, np.array([0, 255]))):
            r = s.poll(sid, timeout_ms=60000)
            assert r is not None and r["status"] == 0 and r["index"] == q
            x = gl[q]
            np.testing.assert_array_equal(r["vis"][chans], oracle.correlate(np.ascontiguousarray(x[:, chans, :])))
            lat[sid].append(r["latency_ms"])
            s.release(sid, q)
    s.close()
    print("\nlatency ms: large", [round(v, 1) for v in lat[a]], "small", [round(v, 1) for v in lat[b]])
    assert max(lat[b]) < 0.5 * min(lat[a]), lat
