"""The first-fit allocator behind footprint admission (CPU)."""
import gen
from paper_1908_09378_gb300.serve import FirstFit


def test_first_fit_alloc_free_coalesce():
    a = FirstFit(4096)
    x = a.alloc(1000)
    y = a.alloc(1000)
    z = a.alloc(1000)
    assert (x, y, z) == (0, 1024, 2048)
    assert a.alloc(2000) is None          # only 1024 left at the end
    a.free(y, 1000)
    assert a.alloc(1024) == 1024          # reuses the hole
    a.free(x, 1000)
    a.free(1024, 1024)
    a.free(z, 1000)
    assert a.starts == [0] and a.lens == [4096] and a.used == 0


def test_first_fit_random_never_overlaps():
    st = gen.Stream(5)
    a = FirstFit(1 << 20)
    live = {}
    for step in range(3000):
        if live and st.uniform(0, 2) == 0:
            off = list(live)[st.uniform(0, len(live) - 1)]
            a.free(off, live.pop(off))
        else:
            n = st.uniform(1, 1 << 14)
            off = a.alloc(n)
            if off is not None:
                rounded = (n + 255) // 256 * 256
                for o, m in live.items():
                    mr = (m + 255) // 256 * 256
                    assert off + rounded <= o or o + mr <= off
                live[off] = n
    for off in list(live):
        a.free(off, live.pop(off))
    assert a.starts == [0] and a.lens == [1 << 20]
