"""Host-side logic of the serving loop (no GPU): the arena's range allocator and the
split of a finished wave's result copies over the copy threads."""
import numpy as np

from paper_2104_14547_gb300 import serve


def test_copy_chunks_cover_every_evaluation_once_in_order():
    rng = np.random.default_rng(3)
    for _ in range(200):
        n = int(rng.integers(1, 80))
        sizes = rng.integers(1024, 65536, size=n).tolist()
        for workers in (1, 2, 3, 8, 100):
            b = serve.copy_chunks(sizes, workers)
            assert b[0] == 0 and b[-1] == n
            assert all(x < y for x, y in zip(b[:-1], b[1:]))      # contiguous, none empty
            assert len(b) - 1 <= min(workers, n)
            if workers > 1 and n >= workers:
                # no chunk holds much more than its share plus one evaluation
                share = sum(sizes) / workers
                assert max(sum(sizes[x:y]) for x, y in zip(b[:-1], b[1:])) <= share + max(sizes)
    assert serve.copy_chunks([], 8) == [0]
    assert serve.copy_chunks([5], 8) == [0, 1]


def test_range_allocator_first_fit_alignment_and_merge():
    a = serve.RangeAllocator(100)
    x = a.alloc(10)
    y = a.alloc(20, align=16)
    z = a.alloc(30)
    assert x == 0 and y == 16 and z == 36
    assert a.alloc(100) is None                          # admission refused when full
    a.release(y, 20)
    a.release(x, 10)
    assert a.alloc(16) == 0                              # freed ranges merged and reused
    a.release(0, 16)
    a.release(z, 30)
    assert a.available == 100 and a.free == [(0, 100)]
