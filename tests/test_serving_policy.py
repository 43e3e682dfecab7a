"""Admission and batching rule of the serving loop (host logic only, no GPU)."""
import collections

import pytest

from paper_2410_11184_gb300.serve import BatchPolicy, percentile


class R:
    def __init__(self, plan, n_ct, words, level=12, scale=1.0):
        self.plan, self.n_ct, self.words, self.level, self.scale = plan, n_ct, words, level, scale

    def key(self):
        return (self.plan, self.n_ct, self.level, self.scale)


def test_admission_respects_budget_and_arrival_order():
    pol = BatchPolicy(budget_bytes=8 * 100 * 2.0, max_batch_ct=8, work_factor=2.0)  # 100 words fit
    waiting = collections.deque([R("a", 1, 40), R("b", 1, 40), R("a", 1, 40), R("a", 1, 10)])
    admitted = []
    assert pol.admit(waiting, admitted) == []
    # 40 + 40 fit, the third (40) does not: it and everything behind it wait (no overtaking)
    assert [r.plan for r in admitted] == ["a", "b"] and len(waiting) == 2
    assert pol.in_use == pytest.approx(8 * 80 * 2.0)
    pol.release([admitted.pop(0)])
    pol.admit(waiting, admitted)
    assert [r.plan for r in admitted] == ["b", "a", "a"] and not waiting


def test_oversized_requests_are_rejected_not_queued_forever():
    pol = BatchPolicy(budget_bytes=8 * 50, max_batch_ct=4, work_factor=1.0)
    big, wide, ok = R("a", 1, 60), R("a", 5, 10), R("a", 1, 10)
    waiting = collections.deque([big, wide, ok])
    admitted = []
    assert pol.admit(waiting, admitted) == [big, wide]
    assert admitted == [ok]


def test_batches_take_the_oldest_shape_up_to_the_ciphertext_limit():
    pol = BatchPolicy(budget_bytes=1e12, max_batch_ct=4)
    a1, b1, a2, a3, a4, a5 = R("a", 2, 1), R("b", 1, 1), R("a", 1, 1), R("a", 2, 1), R("a", 1, 1), R("a", 1, 1)
    admitted = [a1, b1, a2, a3, a4, a5]
    # oldest shape is (a, 2 ciphertexts): a1 and a3 (4 ciphertexts); (a, 1) is another shape
    assert pol.next_batch(admitted) == [a1, a3]
    assert admitted == [b1, a2, a4, a5]
    assert pol.next_batch(admitted) == [b1]
    assert pol.next_batch(admitted) == [a2, a4, a5]
    assert pol.next_batch(admitted) == [] and admitted == []


def test_release_returns_the_budget():
    pol = BatchPolicy(budget_bytes=1e6, work_factor=3.0)
    rs = [R("a", 1, 100), R("a", 1, 50)]
    pol.admit(collections.deque(rs), [])
    assert pol.in_use == pytest.approx(8 * 150 * 3.0)
    pol.release(rs)
    assert pol.in_use == 0.0


def test_percentile_nearest_rank():
    xs = list(range(1, 101))
    assert percentile(xs, 50) == 50 and percentile(xs, 99) == 99 and percentile(xs, 100) == 100
    assert percentile([7.0], 99) == 7.0
    assert percentile([3, 1, 2], 50) == 2


def test_request_ids_unique_across_threads():
    """submit() may run on many client threads: every request gets its own id."""
    import threading

    from paper_2410_11184_gb300.serve import Request

    ids, lock = [], threading.Lock()

    def make():
        got = [Request("p", 1, 0, 1.0, None, None, 1).rid for _ in range(2000)]
        with lock:
            ids.extend(got)

    ts = [threading.Thread(target=make) for _ in range(8)]
    for t in ts:
        t.start()
    for t in ts:
        t.join()
    assert len(ids) == len(set(ids)) == 16000
