"""Oracle results of the full-size workloads, computed in a background thread.

The int64 oracle needs several minutes of host time for the benchmark
workload; started when full-size tests are collected, it runs while the
other GPU tests do (its C loop releases the GIL), and the full-size tests
wait for it.  Only the test-suite uses this module."""
from __future__ import annotations

import threading

import numpy as np

import oracle
import synth

_LOCK = threading.Lock()
_JOBS: dict[str, tuple[threading.Thread, dict]] = {}

LARGE_N_CHANNELS = np.arange(0, 64, 4)   # 16 channels, spread over the band


def _lwa():
    x = synth.config_voltages("lwa")
    return x, oracle.correlate(x)


def _large_n():
    x = synth.config_voltages("large_n")
    return x, LARGE_N_CHANNELS, oracle.correlate(np.ascontiguousarray(x[:, LARGE_N_CHANNELS, :]))


_MAKERS = {"lwa": _lwa, "large_n": _large_n}


def start(name: str) -> None:
    """Begin computing `name` in the background (once)."""
    with _LOCK:
        if name in _JOBS:
            return
        box: dict = {}

        def run():
            try:
                box["value"] = _MAKERS[name]()
            except BaseException as e:   # re-raised in result()
                box["error"] = e

        th = threading.Thread(target=run, name=f"oracle-{name}", daemon=True)
        _JOBS[name] = (th, box)
        th.start()


def result(name: str):
    """The finished result of `name` (started now if it was not)."""
    start(name)
    th, box = _JOBS[name]
    th.join()
    if "error" in box:
        raise box["error"]
    return box["value"]
