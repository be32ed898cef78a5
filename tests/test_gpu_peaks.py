"""The L2-resident random-gather rate (nr_l2_gather_rate) that bench.py reports the field
kernel's gathers against: positive, 16-byte gathers deliver more bytes than 4-byte ones, and
neither exceeds what 32-byte L2 sectors could carry (every gather touches one sector, and the
GB300's L2 serves fewer than 20 TB/s of them)."""
import pytest

from _util import nrmod

pytestmark = pytest.mark.gpu


def test_l2_gather_rates_are_plausible():
    nr = nrmod()
    r4 = nr.nr_l2_gather_rate(0, 32 << 20, 4)
    r16 = nr.nr_l2_gather_rate(0, 32 << 20, 16)
    print(f"L2-resident gathers: 4 B {r4 / 1e9:.0f} GB/s, 16 B {r16 / 1e9:.0f} GB/s")
    assert 0 < r4 < r16
    assert r4 * 8 < 20e12 and r16 * 2 < 20e12     # sectors per second times 32 bytes
