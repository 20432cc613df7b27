"""CCSDS Orbit Mean-Elements Messages (host functions of the library; no GPU).

Pins: keyword values of hand-made KVN and XML messages converted to the units of
sgp4_init, the epoch against Python's own calendar arithmetic (datetime), the two
encodings agreeing, multi-message texts with comments, units and the day-of-year epoch
form, rejection of messages that are incomplete, malformed or of another theory, frame
or time system, the writer/reader round trip, and agreement with the two-line-set
reader on the same element set.
"""
from __future__ import annotations

import math
from datetime import datetime, timedelta

import numpy as np
import pytest

from paper_2603_27830_b300 import omm, tle

JD_2000_NOON = 2451545.0        # Julian date of 2000-01-01 12:00 UT
DEG = math.pi / 180.0
REV_PER_DAY = 2.0 * math.pi / 1440.0


def _jd(dt: datetime) -> float:
    return (dt - datetime(2000, 1, 1, 12)) / timedelta(days=1) + JD_2000_NOON


KVN = """CCSDS_OMM_VERS = 2.0
COMMENT a hand-made message
CREATION_DATE = 2026-01-14T00:00:00
ORIGINATOR = TEST
OBJECT_NAME = TESTSAT
OBJECT_ID = 2026-001A
CENTER_NAME = EARTH
REF_FRAME = TEME
TIME_SYSTEM = UTC
MEAN_ELEMENT_THEORY = SGP4
EPOCH = 2026-01-13T18:00:00.000000
MEAN_MOTION = 15.06000000 [rev/day]
ECCENTRICITY = .0001234
INCLINATION = 53.0000 [deg]
RA_OF_ASC_NODE = 123.4567 [deg]
ARG_OF_PERICENTER = 270.0000 [deg]
MEAN_ANOMALY = 90.0000 [deg]
EPHEMERIS_TYPE = 0
CLASSIFICATION_TYPE = U
NORAD_CAT_ID = 12345
ELEMENT_SET_NO = 999
REV_AT_EPOCH = 0
BSTAR = 0.12345E-3 [1/ER]
MEAN_MOTION_DOT = 0
MEAN_MOTION_DDOT = 0
"""

XML = """<?xml version="1.0" encoding="UTF-8"?>
<ndm>
 <omm id="CCSDS_OMM_VERS" version="2.0">
  <header><CREATION_DATE>2026-01-14T00:00:00</CREATION_DATE><ORIGINATOR>TEST</ORIGINATOR></header>
  <body><segment>
   <metadata>
    <OBJECT_NAME>TESTSAT</OBJECT_NAME><OBJECT_ID>2026-001A</OBJECT_ID>
    <CENTER_NAME>EARTH</CENTER_NAME><REF_FRAME>TEME</REF_FRAME>
    <TIME_SYSTEM>UTC</TIME_SYSTEM><MEAN_ELEMENT_THEORY>SGP4</MEAN_ELEMENT_THEORY>
   </metadata>
   <data>
    <meanElements>
     <EPOCH>2026-01-13T18:00:00.000000</EPOCH>
     <MEAN_MOTION units="rev/day">15.06000000</MEAN_MOTION>
     <ECCENTRICITY>.0001234</ECCENTRICITY>
     <INCLINATION units="deg">53.0000</INCLINATION>
     <RA_OF_ASC_NODE units="deg">123.4567</RA_OF_ASC_NODE>
     <ARG_OF_PERICENTER units="deg">270.0000</ARG_OF_PERICENTER>
     <MEAN_ANOMALY units="deg">90.0000</MEAN_ANOMALY>
    </meanElements>
    <tleParameters>
     <EPHEMERIS_TYPE>0</EPHEMERIS_TYPE><CLASSIFICATION_TYPE>U</CLASSIFICATION_TYPE>
     <NORAD_CAT_ID>12345</NORAD_CAT_ID><ELEMENT_SET_NO>999</ELEMENT_SET_NO>
     <REV_AT_EPOCH>0</REV_AT_EPOCH><BSTAR units="1/ER">0.12345E-3</BSTAR>
     <MEAN_MOTION_DOT>0</MEAN_MOTION_DOT><MEAN_MOTION_DDOT>0</MEAN_MOTION_DDOT>
    </tleParameters>
   </data>
  </segment></body>
 </omm>
</ndm>
"""


def _expected():
    el = np.array([15.06 * REV_PER_DAY, 0.0001234, 53.0 * DEG, 123.4567 * DEG, 270.0 * DEG,
                   90.0 * DEG, 0.12345e-3])
    return el, _jd(datetime(2026, 1, 13, 18))


@pytest.mark.parametrize("text", [KVN, XML], ids=["kvn", "xml"])
def test_fields_units_and_epoch(text):
    s = omm.parse_text(text)
    assert len(s.elements) == 1 and s.rejected == 0
    el, jd = _expected()
    assert np.allclose(s.elements[0], el, rtol=1e-15, atol=0.0)
    assert s.epoch_day[0] + s.epoch_frac[0] == pytest.approx(jd, abs=1e-9)
    assert 0.0 <= s.epoch_frac[0] < 1.0
    assert s.satnum[0] == 12345


def test_kvn_and_xml_agree_exactly():
    a, b = omm.parse_text(KVN), omm.parse_text(XML)
    assert np.array_equal(a.elements, b.elements)
    assert np.array_equal(a.epoch_day, b.epoch_day) and np.array_equal(a.epoch_frac, b.epoch_frac)


def test_several_messages_epoch_forms_and_missing_catalogue_number():
    second = (KVN.replace("EPOCH = 2026-01-13T18:00:00.000000", "EPOCH = 2024-366T23:59:30Z")
                 .replace("NORAD_CAT_ID = 12345\n", "")
                 .replace("COMMENT a hand-made message", "COMMENT leap-year day 366"))
    third = KVN.replace("EPOCH = 2026-01-13T18:00:00.000000", "EPOCH = 2000-03-01")
    s = omm.parse_text(KVN + "\n" + second + third)
    assert len(s.elements) == 3 and s.rejected == 0
    jds = s.epoch_day + s.epoch_frac
    assert jds[0] == pytest.approx(_jd(datetime(2026, 1, 13, 18)), abs=1e-9)
    assert jds[1] == pytest.approx(_jd(datetime(2024, 12, 31, 23, 59, 30)), abs=1e-9)
    assert jds[2] == pytest.approx(_jd(datetime(2000, 3, 1)), abs=1e-9)
    assert list(s.satnum) == [12345, -1, 12345]
    xml3 = XML.replace("</ndm>", "") + "".join(
        XML[XML.index("<omm"):XML.index("</ndm>")] for _ in range(2)) + "</ndm>\n"
    assert len(omm.parse_text(xml3).elements) == 3


@pytest.mark.parametrize("edit", [
    ("BSTAR = 0.12345E-3 [1/ER]\n", ""),                                  # missing keyword
    ("MEAN_ELEMENT_THEORY = SGP4", "MEAN_ELEMENT_THEORY = DSST"),         # another theory
    ("REF_FRAME = TEME", "REF_FRAME = GCRF"),                             # another frame
    ("TIME_SYSTEM = UTC", "TIME_SYSTEM = TAI"),                           # another time system
    ("ECCENTRICITY = .0001234", "ECCENTRICITY = 1.2.3"),                  # malformed number
    ("INCLINATION = 53.0000", "INCLINATION = 53,0000"),                   # decimal comma
    ("EPOCH = 2026-01-13T18:00:00.000000", "EPOCH = 2026-02-30T00:00:00"),  # no such date
    ("EPOCH = 2026-01-13T18:00:00.000000", "EPOCH = 2026-01-13T24:00:00"),  # no such hour
    ("NORAD_CAT_ID = 12345", "NORAD_CAT_ID = 12A45"),                     # malformed number
], ids=["missing", "theory", "frame", "time", "number", "comma", "date", "hour", "catid"])
def test_rejected_messages(edit):
    bad = KVN.replace(*edit)
    assert bad != KVN
    s = omm.parse_text(KVN + bad + KVN)
    assert len(s.elements) == 2 and s.rejected == 1


def test_round_trip():
    rng = np.random.default_rng(5)
    n = 200
    el = np.column_stack([rng.uniform(1.0, 16.5, n) * REV_PER_DAY, rng.uniform(0.0, 0.9, n),
                          rng.uniform(0.0, math.pi, n), rng.uniform(0.0, 2 * math.pi, (n, 3)),
                          rng.uniform(-1e-2, 1e-2, n)])
    day = rng.integers(2415021, 2488070, n).astype(np.int32)      # 1900 .. 2099
    frac = rng.uniform(0.0, 1.0, n)
    text = "".join(omm.format_messages(el, day, frac, np.arange(n)))
    s = omm.parse_text(text)
    assert len(s.elements) == n and s.rejected == 0
    # 17 significant digits and the unit conversions: a few ulp
    assert np.allclose(s.elements, el, rtol=4e-16, atol=1e-300)
    # the epoch is written to the microsecond
    d = (s.epoch_day - day).astype(np.float64) + (s.epoch_frac - frac)
    assert np.abs(d).max() <= 0.51e-6 / 86400.0 + 1e-15
    assert list(s.satnum) == list(range(n))


def test_same_set_as_the_two_line_reader():
    l1 = "1 12345U 26001A   26013.75000000  .00000000  00000-0  12345-3 0  9990"
    l2 = "2 12345  53.0000 123.4567 0001234 270.0000  90.0000 15.06000000    00"

    def fix(line):
        body = line[:68]
        return body + str(sum(int(c) if c.isdigit() else (1 if c == "-" else 0)
                              for c in body) % 10)
    t = tle.parse(fix(l1), fix(l2))
    o = omm.parse_text(KVN)
    assert np.allclose(o.elements, t.elements, rtol=1e-15, atol=0.0)
    assert o.epoch_day[0] == t.epoch_day[0]
    assert o.epoch_frac[0] == pytest.approx(t.epoch_frac[0], abs=1e-12)
    assert o.satnum[0] == t.satnum[0]


def test_bad_arguments():
    from paper_2603_27830_b300 import _lib
    lib = _lib.load()
    assert lib.sgp4_omm_parse_text(None, 0, 0, None, None, None, None, None) == -1
    assert lib.sgp4_omm_parse_text(b"x", 1, 1, None, None, None, None, None) == -1
    with pytest.raises(_lib.Sgp4Error):
        omm.format_messages(np.full((1, 7), np.nan), 2461000, 0.25)
    with pytest.raises(_lib.Sgp4Error):
        omm.format_messages(np.zeros((1, 7)), 2461000, 1.0)
