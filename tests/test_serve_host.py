"""Admission logic of the serving engine (host only): arrival order is kept
and a wave never exceeds the device-memory budget."""
import collections

import pytest


def _engine(budget, in_use=0, max_wave=100):
    pytest.importorskip("torch")
    from paper_2408_06213_gb300 import serve

    e = serve.ServeEngine.__new__(serve.ServeEngine)
    e.hbm_budget, e.in_use, e.max_wave = budget, in_use, max_wave
    e.max_n, e.max_m = 10 ** 7, 10 ** 4
    e.waiting = collections.deque()
    return e, serve


def test_admission_fifo_and_budget():
    e, serve = _engine(budget=20_000)
    reqs = [serve.Request(i, serve.SHUFFLE, 1000) for i in range(12)]  # 8064 bytes each
    for r in reqs:
        e.submit(r)
    wave = e._admit(None)
    assert [r.rid for r in wave] == [0, 1]
    assert sum(r.device_bytes() for r in wave) <= 20_000
    assert [r.rid for r in e.waiting][:2] == [2, 3]


def test_admission_waits_for_memory():
    e, serve = _engine(budget=10_000, in_use=9_000)
    e.submit(serve.Request(0, serve.SAMPLE, 10 ** 6, 1000))  # 4064 bytes
    assert e._admit(None) == []
    e.in_use = 0
    assert [r.rid for r in e._admit(None)] == [0]


def test_admission_rejects_oversized_request():
    e, serve = _engine(budget=1000)
    e.submit(serve.Request(0, serve.SHUFFLE, 10 ** 6))
    with pytest.raises(RuntimeError):
        e._admit(None)


def test_admission_wave_cap():
    e, serve = _engine(budget=10 ** 9, max_wave=5)
    for i in range(9):
        e.submit(serve.Request(i, serve.SAMPLE, 100, 3))
    assert len(e._admit(None)) == 5 and len(e.waiting) == 4


def test_submit_refuses_requests_beyond_the_reserved_limits():
    e, serve = _engine(budget=10 ** 12)
    with pytest.raises(ValueError):
        e.submit(serve.Request(0, serve.SHUFFLE, 10 ** 7 + 1))
    with pytest.raises(ValueError):
        e.submit(serve.Request(1, serve.SAMPLE, 10 ** 8, 10 ** 4 + 1))
    e.submit(serve.Request(2, serve.SHUFFLE, 10 ** 7))
    e.submit(serve.Request(3, serve.SAMPLE, 10 ** 8, 10 ** 4))
    assert [r.rid for r in e.waiting] == [2, 3]
