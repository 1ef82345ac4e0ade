"""Host-side arena manager of the serving loop (dseed_arena_*), checked against
an independent model of first-fit allocation over a sorted free list."""
import numpy as np
import pytest

from paper_2410_16727_gb300 import binding as B
from paper_2410_16727_gb300 import build as BLD


@pytest.fixture(scope="module", autouse=True)
def lib():
    try:
        BLD.build()
    except RuntimeError as e:  # pragma: no cover
        pytest.skip(str(e))
    B._lib = None
    return B.load()


class Model:
    """First fit over free intervals kept sorted by start; merge on free."""

    def __init__(self, size):
        self.free = [(0, size)]
        self.taken = {}

    def alloc(self, n):
        n = max(1, n)
        n = (n + 255) // 256 * 256
        for i, (o, s) in enumerate(self.free):
            if s >= n:
                if s == n:
                    self.free.pop(i)
                else:
                    self.free[i] = (o + n, s - n)
                self.taken[o] = n
                return o
        return None

    def release(self, o):
        n = self.taken.pop(o)
        self.free.append((o, n))
        self.free.sort()
        merged = []
        for a, s in self.free:
            if merged and merged[-1][0] + merged[-1][1] == a:
                merged[-1] = (merged[-1][0], merged[-1][1] + s)
            else:
                merged.append((a, s))
        self.free = merged


def test_alignment_reuse_and_merge():
    a = B.Arena(10 * 256)
    o1, o2, o3 = a.alloc(1), a.alloc(300), a.alloc(256)
    assert (o1, o2, o3) == (0, 256, 768)
    assert a.usage()[0] == 4 * 256
    a.free(o2)
    assert a.alloc(512) == 256          # first fit reuses the hole
    a.free(256)
    a.free(o1)
    a.free(o3)
    assert a.usage()[0] == 0 and a.usage()[2] == 10 * 256   # everything merged back
    assert a.usage()[1] == 4 * 256                           # peak kept


def test_out_of_memory_and_bad_free():
    a = B.Arena(4096)
    assert a.alloc(4097) is None
    o = a.alloc(4096)
    assert o == 0 and a.alloc(1) is None
    with pytest.raises(B.DseedError, match="not an allocated block"):
        a.free(128)


def test_random_sequence_matches_model():
    rng = np.random.default_rng(0)
    size = 1 << 20
    a, m = B.Arena(size), Model(size)
    live = []
    for step in range(3000):
        if live and rng.random() < 0.45:
            o = live.pop(int(rng.integers(0, len(live))))
            a.free(o)
            m.release(o)
        else:
            n = int(rng.integers(1, 40000))
            got, want = a.alloc(n), m.alloc(n)
            assert got == want
            if got is not None:
                live.append(got)
        used = sum(m.taken.values())
        assert a.usage()[0] == used
        assert a.usage()[2] == max([s for _, s in m.free], default=0)
