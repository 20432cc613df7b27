// CCSDS Orbit Mean-Elements Messages (host code): read the SGP4 mean elements and epoch
// of OMMs in their two encodings, KVN (keyword = value lines) and XML, into the
// elements and split epoch that sgp4_init takes, and write KVN messages (synthetic
// catalogues).  The OMM is the standard successor of the two-line set for the same
// element sets (the paper's catalogue source, Sec. 3.1); it carries the epoch as a
// calendar date and time, kept here as a split Julian date (Sec. 6).
//
// Keywords read (CCSDS 502.0-B, OMM with MEAN_ELEMENT_THEORY = SGP4):
//   EPOCH               UTC, "YYYY-MM-DDThh:mm:ss[.f]" or "YYYY-DDDThh:mm:ss[.f]"
//                       (a trailing 'Z' and a date without a time are accepted)
//   MEAN_MOTION         rev/day (Kozai, as in the two-line set)
//   ECCENTRICITY, INCLINATION, RA_OF_ASC_NODE, ARG_OF_PERICENTER, MEAN_ANOMALY (deg)
//   BSTAR               1/Earth radii
//   NORAD_CAT_ID        optional integer (-1 when absent)
//   MEAN_ELEMENT_THEORY, REF_FRAME, TIME_SYSTEM: optional; if present they must be
//                       SGP4 (or SGP/SGP4), TEME and UTC, else the message is rejected
// KVN: a message starts at each CCSDS_OMM_VERS line (a text without one is one
// message); COMMENT lines and other keywords are skipped; a value may carry a
// "[units]" suffix.  XML: one message per <omm> element (an <ndm> container or none
// around them); a keyword's value is the text of the first element of that name.
// Numbers: decimal with optional exponent, in the C locale.
#include <cctype>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>

#include "sgp4.h"

namespace {

constexpr double kPi = 3.14159265358979323846;
constexpr double kDeg = kPi / 180.0;
constexpr double kRevPerDayToRadPerMin = 2.0 * kPi / 1440.0;

enum Key { kEpoch, kMeanMotion, kEcc, kIncl, kRaan, kArgp, kMa, kBstar, kCatId, kTheory,
           kFrame, kTimeSystem, kNumKeys };
const char* const kKeyName[kNumKeys] = {
    "EPOCH", "MEAN_MOTION", "ECCENTRICITY", "INCLINATION", "RA_OF_ASC_NODE",
    "ARG_OF_PERICENTER", "MEAN_ANOMALY", "BSTAR", "NORAD_CAT_ID", "MEAN_ELEMENT_THEORY",
    "REF_FRAME", "TIME_SYSTEM"};

struct Message {
  std::string value[kNumKeys];
  bool has[kNumKeys] = {};
  bool any = false;
};

std::string trim(const std::string& s) {
  size_t a = 0, b = s.size();
  while (a < b && std::isspace((unsigned char)s[a])) ++a;
  while (b > a && std::isspace((unsigned char)s[b - 1])) --b;
  return s.substr(a, b - a);
}

std::string upper(std::string s) {
  for (char& c : s) c = (char)std::toupper((unsigned char)c);
  return s;
}

int key_index(const std::string& k) {
  for (int q = 0; q < kNumKeys; ++q)
    if (k == kKeyName[q]) return q;
  return -1;
}

// A whole-string decimal number (optional sign, exponent).
bool parse_real(const std::string& s, double* out) {
  if (s.empty()) return false;
  for (char c : s)
    if (!(std::isdigit((unsigned char)c) || c == '+' || c == '-' || c == '.' || c == 'e' ||
          c == 'E'))
      return false;
  char* end = nullptr;
  const double v = std::strtod(s.c_str(), &end);
  if (end != s.c_str() + s.size() || !std::isfinite(v)) return false;
  *out = v;
  return true;
}

bool parse_int(const std::string& s, long long lo, long long hi, long long* out) {
  if (s.empty() || s.size() > 18) return false;
  size_t k = 0;
  bool neg = false;
  if (s[0] == '+' || s[0] == '-') { neg = s[0] == '-'; k = 1; }
  if (k == s.size()) return false;
  long long v = 0;
  for (; k < s.size(); ++k) {
    if (!std::isdigit((unsigned char)s[k])) return false;
    v = v * 10 + (s[k] - '0');
  }
  v = neg ? -v : v;
  if (v < lo || v > hi) return false;
  *out = v;
  return true;
}

// Julian day number (the Julian date at noon) of a Gregorian calendar date, by the
// integer formula of Fliegel and Van Flandern (1968).
long long julian_day_number(long long y, long long m, long long d) {
  const long long a = (m - 14) / 12;
  return (1461 * (y + 4800 + a)) / 4 + (367 * (m - 2 - 12 * a)) / 12 -
         (3 * ((y + 4900 + a) / 100)) / 4 + d - 32075;
}

bool leap(long long y) { return (y % 4 == 0 && y % 100 != 0) || y % 400 == 0; }

int days_in_month(long long y, int m) {
  static const int kDays[12] = {31, 28, 31, 30, 31, 30, 31, 31, 30, 31, 30, 31};
  return m == 2 && leap(y) ? 29 : kDays[m - 1];
}

bool digits(const std::string& s, size_t at, size_t n, long long* out) {
  if (at + n > s.size()) return false;
  long long v = 0;
  for (size_t k = at; k < at + n; ++k) {
    if (!std::isdigit((unsigned char)s[k])) return false;
    v = v * 10 + (s[k] - '0');
  }
  *out = v;
  return true;
}

// ISO 8601 epoch (UTC) -> Julian date as day + fraction in [0, 1), the convention of
// sgp4_tle_parse (0h of a date is JDN - 0.5).  Years 1583 .. 9999.
bool parse_epoch(std::string s, int32_t* day, double* frac) {
  if (!s.empty() && (s.back() == 'Z' || s.back() == 'z')) s.pop_back();
  long long y, m = 1, d = 1, doy = 0;
  if (!digits(s, 0, 4, &y) || y < 1583 || s.size() < 8 || s[4] != '-') return false;
  size_t p;
  if (s.size() >= 10 && s[7] == '-') {                     // YYYY-MM-DD
    if (!digits(s, 5, 2, &m) || !digits(s, 8, 2, &d)) return false;
    if (m < 1 || m > 12 || d < 1 || d > days_in_month(y, (int)m)) return false;
    p = 10;
  } else {                                                 // YYYY-DDD
    if (!digits(s, 5, 3, &doy) || doy < 1 || doy > (leap(y) ? 366 : 365)) return false;
    p = 8;
  }
  double secs = 0.0;
  if (p < s.size()) {
    if (s[p] != 'T' && s[p] != 't') return false;
    long long hh, mi;
    if (!digits(s, p + 1, 2, &hh) || s.size() < p + 6 || s[p + 3] != ':' ||
        !digits(s, p + 4, 2, &mi) || hh > 23 || mi > 59)
      return false;
    double ss = 0.0;
    if (p + 6 < s.size()) {
      if (s[p + 6] != ':') return false;
      const std::string sec = s.substr(p + 7);
      if (sec.size() < 2 || !std::isdigit((unsigned char)sec[0]) ||
          !std::isdigit((unsigned char)sec[1]) || !parse_real(sec, &ss) || ss < 0.0 ||
          ss >= 61.0)
        return false;
    }
    secs = (double)(hh * 3600 + mi * 60) + ss;
  }
  long long jdn = doy > 0 ? julian_day_number(y, 1, 1) + doy - 1 : julian_day_number(y, m, d);
  long long dd = jdn - 1;
  double f = 0.5 + secs / 86400.0;
  while (f >= 1.0) { dd += 1; f -= 1.0; }
  if (dd < INT32_MIN || dd > INT32_MAX) return false;
  *day = (int32_t)dd;
  *frac = f;
  return true;
}

// Message -> elements; false if a required keyword is missing or malformed, or the
// theory, frame or time system is not the one of these elements.
bool to_elements(const Message& m, double* el, int32_t* eday, double* efrac, int32_t* num) {
  static const int kReq[] = {kEpoch, kMeanMotion, kEcc, kIncl, kRaan, kArgp, kMa, kBstar};
  for (int q : kReq)
    if (!m.has[q]) return false;
  if (m.has[kTheory]) {
    const std::string t = upper(m.value[kTheory]);
    if (t != "SGP4" && t != "SGP/SGP4") return false;
  }
  if (m.has[kFrame] && upper(m.value[kFrame]) != "TEME") return false;
  if (m.has[kTimeSystem] && upper(m.value[kTimeSystem]) != "UTC") return false;
  double mm, e, inc, raan, argp, ma, bstar;
  if (!parse_real(m.value[kMeanMotion], &mm) || !parse_real(m.value[kEcc], &e) ||
      !parse_real(m.value[kIncl], &inc) || !parse_real(m.value[kRaan], &raan) ||
      !parse_real(m.value[kArgp], &argp) || !parse_real(m.value[kMa], &ma) ||
      !parse_real(m.value[kBstar], &bstar))
    return false;
  int32_t day;
  double frac;
  if (!parse_epoch(m.value[kEpoch], &day, &frac)) return false;
  long long id = -1;
  if (m.has[kCatId] && !parse_int(m.value[kCatId], 0, INT32_MAX, &id)) return false;
  el[0] = mm * kRevPerDayToRadPerMin;
  el[1] = e;
  el[2] = inc * kDeg;
  el[3] = raan * kDeg;
  el[4] = argp * kDeg;
  el[5] = ma * kDeg;
  el[6] = bstar;
  *eday = day;
  *efrac = frac;
  *num = (int32_t)id;
  return true;
}

// Appends the messages of a KVN text to `out` through `emit`.
template <class Emit>
void read_kvn(const char* text, size_t len, Emit emit) {
  Message cur;
  size_t a = 0;
  while (a < len) {
    size_t b = a;
    while (b < len && text[b] != '\n') ++b;
    const std::string line = trim(std::string(text + a, b - a));
    a = b + 1;
    if (line.empty() || line.compare(0, 7, "COMMENT") == 0) continue;
    const size_t eq = line.find('=');
    if (eq == std::string::npos) continue;
    const std::string key = upper(trim(line.substr(0, eq)));
    std::string val = trim(line.substr(eq + 1));
    const size_t br = val.find('[');
    if (br != std::string::npos) val = trim(val.substr(0, br));
    if (key == "CCSDS_OMM_VERS") {
      if (cur.any) emit(cur);
      cur = Message();
      cur.any = true;
      continue;
    }
    const int q = key_index(key);
    if (q >= 0 && !cur.has[q]) {
      cur.value[q] = val;
      cur.has[q] = true;
      cur.any = true;
    }
  }
  if (cur.any) emit(cur);
}

// Position just past the start tag <name ...> at or after `from` in [from, end), or npos.
size_t find_start_tag(const std::string& s, const std::string& name, size_t from, size_t end,
                      size_t* tag_at) {
  const std::string open = "<" + name;
  size_t p = from;
  while ((p = s.find(open, p)) != std::string::npos && p < end) {
    const size_t q = p + open.size();
    if (q < s.size() && (s[q] == '>' || s[q] == '/' || std::isspace((unsigned char)s[q]))) {
      const size_t gt = s.find('>', q);
      if (gt == std::string::npos || gt >= end) return std::string::npos;
      if (tag_at) *tag_at = p;
      return s[gt - 1] == '/' ? std::string::npos : gt + 1;   // <name/> has no value
    }
    p = q;
  }
  return std::string::npos;
}

template <class Emit>
void read_xml(const char* text, size_t len, Emit emit) {
  const std::string s(text, len);
  auto read_block = [&](size_t from, size_t end) {
    Message m;
    for (int q = 0; q < kNumKeys; ++q) {
      const size_t v = find_start_tag(s, kKeyName[q], from, end, nullptr);
      if (v == std::string::npos) continue;
      const size_t close = s.find("</" + std::string(kKeyName[q]), v);
      if (close == std::string::npos || close > end) continue;
      m.value[q] = trim(s.substr(v, close - v));
      m.has[q] = true;
      m.any = true;
    }
    if (m.any) emit(m);
  };
  size_t pos = 0, tag = 0;
  bool found = false;
  size_t body;
  while ((body = find_start_tag(s, "omm", pos, s.size(), &tag)) != std::string::npos) {
    found = true;
    size_t end = s.find("</omm", body);
    if (end == std::string::npos) end = s.size();
    read_block(body, end);
    pos = end;
  }
  if (!found) read_block(0, s.size());
}

// Gregorian calendar date of a Julian day number (the inverse of julian_day_number,
// Fliegel and Van Flandern).
void calendar(long long jdn, long long* y, long long* m, long long* d) {
  long long l = jdn + 68569;
  const long long n = 4 * l / 146097;
  l = l - (146097 * n + 3) / 4;
  const long long i = 4000 * (l + 1) / 1461001;
  l = l - 1461 * i / 4 + 31;
  const long long j = 80 * l / 2447;
  *d = l - 2447 * j / 80;
  l = j / 11;
  *m = j + 2 - 12 * l;
  *y = 100 * (n - 49) + i + l;
}

}  // namespace

extern "C" int64_t sgp4_omm_parse_text(const char* text, size_t len, int64_t capacity,
                                       double* elements, int32_t* epoch_day, double* epoch_frac,
                                       int32_t* satnum, int64_t* n_rejected) {
  if (!text || capacity < 0 || (capacity > 0 && (!elements || !epoch_day || !epoch_frac)))
    return -1;
  int64_t count = 0, rejected = 0;
  auto emit = [&](const Message& m) {
    double el[7];
    int32_t day, num;
    double frac;
    if (!to_elements(m, el, &day, &frac, &num)) { ++rejected; return; }
    if (count < capacity) {
      for (int k = 0; k < 7; ++k) elements[count * 7 + k] = el[k];
      epoch_day[count] = day;
      epoch_frac[count] = frac;
      if (satnum) satnum[count] = num;
    }
    ++count;
  };
  size_t k = 0;
  while (k < len && std::isspace((unsigned char)text[k])) ++k;
  if (k < len && text[k] == '<') read_xml(text, len, emit);
  else read_kvn(text, len, emit);
  if (n_rejected) *n_rejected = rejected;
  return count;
}

extern "C" sgp4_result sgp4_omm_format(const double* elements, int32_t epoch_day,
                                       double epoch_frac, int32_t satnum, const char* name,
                                       char* buf, size_t cap) {
  if (!elements || !buf || cap == 0) return SGP4_ERR_ARG;
  if (!(epoch_frac >= 0.0 && epoch_frac < 1.0)) return SGP4_ERR_ARG;
  for (int k = 0; k < 7; ++k)
    if (!std::isfinite(elements[k])) return SGP4_ERR_ARG;
  if (name && (std::strchr(name, '\n') || std::strchr(name, '\r'))) return SGP4_ERR_ARG;
  // epoch: Julian date day + frac = JDN - 0.5 + time of day
  long long jdn = (long long)epoch_day + 1;
  double tod = epoch_frac - 0.5;
  if (tod < 0.0) { tod += 1.0; jdn -= 1; }
  long long us = std::llround(tod * 86400.0e6);            // microseconds of the day
  if (us >= 86400LL * 1000000) { us -= 86400LL * 1000000; jdn += 1; }
  long long y, mo, d;
  calendar(jdn, &y, &mo, &d);
  if (y < 1583 || y > 9999) return SGP4_ERR_ARG;
  const long long hh = us / 3600000000LL, mi = us / 60000000LL % 60, ss = us / 1000000 % 60;
  const long long frac_us = us % 1000000;
  char idbuf[32];
  if (satnum >= 0) std::snprintf(idbuf, sizeof idbuf, "%d", satnum);
  const int w = std::snprintf(
      buf, cap,
      "CCSDS_OMM_VERS = 2.0\n"
      "CREATION_DATE = %04lld-%02lld-%02lldT%02lld:%02lld:%02lld.%06lld\n"
      "ORIGINATOR = SGP4-B300\n"
      "OBJECT_NAME = %s\n"
      "OBJECT_ID = %s\n"
      "CENTER_NAME = EARTH\n"
      "REF_FRAME = TEME\n"
      "TIME_SYSTEM = UTC\n"
      "MEAN_ELEMENT_THEORY = SGP4\n"
      "EPOCH = %04lld-%02lld-%02lldT%02lld:%02lld:%02lld.%06lld\n"
      "MEAN_MOTION = %.17g [rev/day]\n"
      "ECCENTRICITY = %.17g\n"
      "INCLINATION = %.17g [deg]\n"
      "RA_OF_ASC_NODE = %.17g [deg]\n"
      "ARG_OF_PERICENTER = %.17g [deg]\n"
      "MEAN_ANOMALY = %.17g [deg]\n"
      "EPHEMERIS_TYPE = 0\n"
      "CLASSIFICATION_TYPE = U\n"
      "%s%s%s"
      "ELEMENT_SET_NO = 999\n"
      "REV_AT_EPOCH = 0\n"
      "BSTAR = %.17g [1/ER]\n"
      "MEAN_MOTION_DOT = 0 [rev/day**2]\n"
      "MEAN_MOTION_DDOT = 0 [rev/day**3]\n",
      y, mo, d, hh, mi, ss, frac_us, name ? name : "UNNAMED", "UNKNOWN", y,
      mo, d, hh, mi, ss, frac_us, elements[0] / kRevPerDayToRadPerMin, elements[1],
      elements[2] / kDeg, elements[3] / kDeg, elements[4] / kDeg, elements[5] / kDeg,
      satnum >= 0 ? "NORAD_CAT_ID = " : "", satnum >= 0 ? idbuf : "", satnum >= 0 ? "\n" : "",
      elements[6]);
  if (w < 0 || (size_t)w >= cap) return SGP4_ERR_ARG;
  return SGP4_OK;
}
