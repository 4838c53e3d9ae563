"""Host-side logic of the render server (no GPU): how images are split into
row bands, how launches take bands under the ray budget, first come first
served."""
import collections
from dataclasses import dataclass

from paper_1001_2049_b300.serve import plan_bands, take_units


def test_bands_cover_the_image_exactly_once():
    for h, w, budget in [(1080, 1920, 1 << 18), (512, 512, 1 << 18), (7, 3, 5), (1, 1000, 10),
                         (1024, 1024, 0), (300, 200, 200 * 300)]:
        bands = plan_bands(h, w, budget)
        rows = [r for r0, n in bands for r in range(r0, r0 + n)]
        assert rows == list(range(h))
        if budget and h * w > budget:
            assert all(n * w <= max(budget, w) for _, n in bands)
        else:
            assert bands == [(0, h)]


@dataclass
class _U:
    rays: int
    name: str = ""


def test_a_launch_takes_bands_in_order_within_the_budget():
    q = collections.deque(_U(r, str(i)) for i, r in enumerate([100, 50, 80, 30, 500, 10]))
    first = take_units(q, 8, 200)
    assert [u.name for u in first] == ["0", "1"]          # 100 + 50; 80 would pass 200
    second = take_units(q, 8, 200)
    assert [u.name for u in second] == ["2", "3"]
    third = take_units(q, 8, 200)                          # alone over budget: still taken
    assert [u.name for u in third] == ["4"]
    assert [u.name for u in take_units(q, 8, 0)] == ["5"]
    assert not q
    q = collections.deque(_U(1) for _ in range(10))
    assert len(take_units(q, 4, 0)) == 4 and len(q) == 6
