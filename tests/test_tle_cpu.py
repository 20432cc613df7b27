"""Two-line element sets (host functions of the library; no GPU).

Pins: fields read from hand-made lines at the format's columns, the epoch against
Python's own calendar arithmetic (datetime), the checksum rule, rejection of damaged
sets, and the writer/reader round trip at the format's resolution.
"""
from __future__ import annotations

import math
from datetime import datetime, timedelta

import numpy as np
import pytest

from paper_2603_27830_b300 import _lib
from paper_2603_27830_b300 import tle
from paper_2603_27830_b300 import workloads as W

JD_2000_NOON = 2451545.0        # Julian date of 2000-01-01 12:00 UT


def _checksum(s: str) -> str:
    return str(sum(int(c) if c.isdigit() else (1 if c == "-" else 0) for c in s[:68]) % 10)


def _line(body: str) -> str:
    assert len(body) == 68
    return body + _checksum(body)


def _jd(dt: datetime) -> tuple[int, float]:
    days = (dt - datetime(2000, 1, 1, 12)) / timedelta(days=1) + JD_2000_NOON
    return int(math.floor(days)), days - math.floor(days)


L1 = _line("1 12345U 26001A   26013.75000000  .00000000  00000-0  12345-3 0  999")
L2 = _line("2 12345  53.0000 123.4567 0001234 270.0000  90.0000 15.06000000    0")


def test_fields_units_and_epoch():
    s = tle.parse(L1, L2)
    el = s.elements[0]
    assert el[0] == pytest.approx(15.06 * 2 * math.pi / 1440, rel=1e-15)
    assert el[1] == pytest.approx(0.0001234, rel=1e-15)
    np.testing.assert_allclose(el[2:6], np.radians([53.0, 123.4567, 270.0, 90.0]), rtol=1e-15)
    assert el[6] == pytest.approx(0.12345e-3, rel=1e-15)
    assert int(s.satnum[0]) == 12345
    # day 13.75 of 2026 is 2026-01-13 18:00 UT
    day, frac = _jd(datetime(2026, 1, 13, 18))
    assert (int(s.epoch_day[0]), float(s.epoch_frac[0])) == (day, pytest.approx(frac, abs=1e-12))


@pytest.mark.parametrize("yy,year", [("57", 1957), ("99", 1999), ("00", 2000), ("56", 2056)])
def test_two_digit_year_window(yy, year):
    l1 = _line(L1[:18] + yy + "001.50000000" + L1[32:68])
    s = tle.parse(l1, L2)
    day, frac = _jd(datetime(year, 1, 1, 12))
    assert int(s.epoch_day[0]) == day and float(s.epoch_frac[0]) == pytest.approx(frac, abs=1e-12)


def test_bstar_sign_and_exponent_forms():
    for field, want in ((" 12345-3", 0.12345e-3), ("-11606-4", -0.11606e-4),
                        (" 00000+0", 0.0), (" 50000+1", 5.0)):
        l1 = _line(L1[:53] + field + L1[61:68])
        assert tle.parse(l1, L2).elements[0, 6] == pytest.approx(want, rel=1e-15, abs=0)


def test_alpha5_catalogue_number():
    l1 = _line(L1[:2] + "A0001" + L1[7:68])
    l2 = _line(L2[:2] + "A0001" + L2[7:68])
    assert int(tle.parse(l1, l2).satnum[0]) == 100001
    l1 = _line(L1[:2] + "Z9999" + L1[7:68])
    l2 = _line(L2[:2] + "Z9999" + L2[7:68])
    assert int(tle.parse(l1, l2).satnum[0]) == 339999


@pytest.mark.parametrize("damage", ["checksum", "satnum", "short", "swap", "field"])
def test_damaged_sets_are_rejected(damage):
    l1, l2 = L1, L2
    if damage == "checksum":
        l1 = l1[:68] + str((int(l1[68]) + 1) % 10)
    elif damage == "satnum":
        l2 = _line(L2[:2] + "12346" + L2[7:68])
    elif damage == "short":
        l2 = L2[:60]
    elif damage == "swap":
        l1, l2 = L2, L1
    elif damage == "field":
        l2 = _line(L2[:8] + " 53.0x00" + L2[16:68])
    with pytest.raises(_lib.Sgp4Error):
        tle.parse(l1, l2)


def test_text_with_names_blanks_and_a_bad_set():
    bad2 = L2[:68] + str((int(L2[68]) + 3) % 10)
    text = "\n".join(["SAT A", L1, L2, "", L1, bad2, "SAT C", L1 + "\r", L2 + "  ", L1]) + "\n"
    s = tle.parse_text(text)
    assert len(s.satnum) == 2 and s.rejected == 2      # the bad checksum and a lone line 1
    np.testing.assert_array_equal(s.elements[0], s.elements[1])


def test_round_trip_at_format_resolution():
    rng = np.random.default_rng(5)
    el = np.concatenate([W.config2(seed=2, n=300).elements,
                         W.catalogue_elements(rng, 300, invalid_frac=0.0)])
    n = len(el)
    el[:, 6] = np.where(rng.uniform(size=n) < 0.2, -el[:, 6], el[:, 6])
    day = (2461040 + rng.integers(-4000, 4000, n)).astype(np.int32)
    frac = rng.uniform(0.0, 1.0, n)
    sets = tle.format_sets(el, day, frac, satnum=np.arange(n) + 40000)
    for a, b in sets:
        assert len(a) == 69 and len(b) == 69
        assert a[68] == _checksum(a) and b[68] == _checksum(b)
    back = tle.parse_text("\n".join(f"{a}\n{b}" for a, b in sets))
    assert len(back.satnum) == n and back.rejected == 0
    np.testing.assert_array_equal(back.satnum, np.arange(n) + 40000)
    two_pi = 2 * math.pi
    ang = lambda x: np.mod(x, two_pi)  # noqa: E731
    assert np.all(np.abs(back.elements[:, 0] - el[:, 0]) <= 0.5e-8 * two_pi / 1440 * 1.001)
    assert np.all(np.abs(back.elements[:, 1] - el[:, 1]) <= 0.5e-7 * 1.001)
    assert np.all(np.abs(back.elements[:, 2] - el[:, 2]) <= math.radians(0.5e-4) * 1.001)
    for k in (3, 4, 5):
        d = np.abs(ang(back.elements[:, k]) - ang(el[:, k]))
        assert np.all(np.minimum(d, two_pi - d) <= math.radians(0.5e-4) * 1.001)
    np.testing.assert_allclose(back.elements[:, 6], el[:, 6], rtol=0.5e-4 * 1.01, atol=0)
    t_in = (day - 2461000).astype(np.float64) + frac
    t_out = (back.epoch_day - 2461000).astype(np.float64) + back.epoch_frac
    assert np.all(np.abs(t_out - t_in) <= 0.5e-8 * 1.001)
    # the writer reproduces its own lines from what it read
    again = tle.format_sets(back.elements, back.epoch_day, back.epoch_frac, back.satnum)
    assert again == sets
