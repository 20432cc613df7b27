// Two-line element sets (host code): parse the fixed-column NORAD format into the
// elements and split epoch that sgp4_init takes, and format elements back into it
// (synthetic catalogues).  The paper reads its Starlink catalogue from TLEs
// (Sec. 3.1) and stresses a split epoch (Sec. 6).
//
// Columns used (1-based, as the format defines them):
//   line 1: 1 line number '1'; 3-7 catalogue number; 19-20 epoch year (57-99 ->
//           19xx, 00-56 -> 20xx); 21-32 epoch day of year with fraction; 54-61 B*
//           as a signed 5-digit mantissa with an implied leading decimal point and a
//           signed exponent digit; 69 checksum.
//   line 2: 1 '2'; 3-7 catalogue number; 9-16 inclination (deg); 18-25 RAAN (deg);
//           27-33 eccentricity (implied leading decimal point); 35-42 argument of
//           perigee (deg); 44-51 mean anomaly (deg); 53-63 mean motion (rev/day);
//           69 checksum.
// Checksum: the sum of the digits of columns 1-68, each '-' counting 1, modulo 10.
// Epoch: Julian date of 0h January 1 of the year (Gregorian calendar, 1901-2099) plus
// day-of-year - 1, returned as an integer day and a fraction in [0, 1).
#include <cctype>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>

#include "sgp4.h"

namespace {

constexpr double kPi = 3.14159265358979323846;
constexpr double kDeg = kPi / 180.0;
constexpr double kRevPerDayToRadPerMin = 2.0 * kPi / 1440.0;

// Length of a line without trailing CR, LF, spaces.
size_t line_len(const char* s) {
  size_t n = std::strlen(s);
  while (n > 0 && (s[n - 1] == '\n' || s[n - 1] == '\r' || s[n - 1] == ' ')) --n;
  return n;
}

int checksum(const char* s) {
  int sum = 0;
  for (int k = 0; k < 68; ++k) {
    if (s[k] >= '0' && s[k] <= '9') sum += s[k] - '0';
    else if (s[k] == '-') sum += 1;
  }
  return sum % 10;
}

// Field [c0, c1] (1-based inclusive columns) copied to buf with surrounding blanks cut.
bool field(const char* s, int c0, int c1, char* buf, size_t cap) {
  int a = c0 - 1, b = c1 - 1;
  while (a <= b && s[a] == ' ') ++a;
  while (b >= a && s[b] == ' ') --b;
  const int n = b - a + 1;
  if (n <= 0 || (size_t)n >= cap) return false;
  std::memcpy(buf, s + a, (size_t)n);
  buf[n] = '\0';
  return true;
}

// Plain decimal number (optional sign, digits, optional fraction): no exponent, no
// other characters.
bool parse_decimal(const char* t, double* out) {
  const char* p = t;
  bool neg = false;
  if (*p == '+' || *p == '-') neg = *p++ == '-';
  bool digits = false;
  double v = 0.0;
  while (std::isdigit((unsigned char)*p)) { v = v * 10.0 + (*p++ - '0'); digits = true; }
  if (*p == '.') {
    ++p;
    double scale = 1.0;
    long long frac = 0;
    while (std::isdigit((unsigned char)*p)) {
      if (scale < 1e18) { frac = frac * 10 + (*p - '0'); scale *= 10.0; }
      ++p;
      digits = true;
    }
    v += (double)frac / scale;
  }
  if (!digits || *p != '\0') return false;
  *out = neg ? -v : v;
  return true;
}

// Catalogue number: five digits, or "Alpha-5" (a letter for the ten-thousands, I and
// O skipped: A = 10 .. Z = 33, then four digits).
bool parse_satnum(const char* s, int32_t* out) {
  char b[8];
  std::memcpy(b, s + 2, 5);
  b[5] = '\0';
  int lead;
  const char c = b[0];
  if (c >= '0' && c <= '9') lead = c - '0';
  else if (c == ' ') lead = 0;
  else if (c >= 'A' && c <= 'Z' && c != 'I' && c != 'O')
    lead = 10 + (c - 'A') - (c > 'I' ? 1 : 0) - (c > 'O' ? 1 : 0);
  else return false;
  int v = lead;
  for (int k = 1; k < 5; ++k) {
    const char d = b[k] == ' ' ? '0' : b[k];
    if (d < '0' || d > '9') return false;
    v = v * 10 + (d - '0');
  }
  *out = v;
  return true;
}

// Mantissa-exponent field such as " 34123-4" (0.34123e-4) or "-11606-4".
bool parse_exp_field(const char* s, int c0, int c1, double* out) {
  char b[16];
  const int n = c1 - c0 + 1;
  std::memcpy(b, s + c0 - 1, (size_t)n);
  b[n] = '\0';
  int k = 0;
  while (b[k] == ' ') ++k;
  bool neg = false;
  if (b[k] == '-' || b[k] == '+') neg = b[k++] == '-';
  long long mant = 0;
  int nd = 0;
  while (b[k] >= '0' && b[k] <= '9') { mant = mant * 10 + (b[k++] - '0'); ++nd; }
  if (nd == 0) return false;
  int ex = 0;
  if (b[k] == '-' || b[k] == '+') {
    const bool eneg = b[k++] == '-';
    if (b[k] < '0' || b[k] > '9') return false;
    ex = b[k++] - '0';
    if (eneg) ex = -ex;
  }
  while (b[k] == ' ') ++k;
  if (b[k] != '\0') return false;
  const double v = (double)mant / std::pow(10.0, nd) * std::pow(10.0, ex);
  *out = neg ? -v : v;
  return true;
}

// Julian date of 0h January 1 of `year` is jan1(year) + 0.5 (valid 1901-2099).
long long jan1(int year) { return 367LL * year - (7LL * year) / 4 + 31 + 1721013; }

}  // namespace

extern "C" sgp4_result sgp4_tle_parse(const char* line1, const char* line2, double* elements,
                                      int32_t* epoch_day, double* epoch_frac, int32_t* satnum) {
  if (!line1 || !line2 || !elements || !epoch_day || !epoch_frac) return SGP4_ERR_ARG;
  if (line_len(line1) < 69 || line_len(line2) < 69) return SGP4_ERR_ARG;
  if (line1[0] != '1' || line2[0] != '2') return SGP4_ERR_ARG;
  if (checksum(line1) != line1[68] - '0' || checksum(line2) != line2[68] - '0') return SGP4_ERR_ARG;
  int32_t n1 = 0, n2 = 0;
  if (!parse_satnum(line1, &n1) || !parse_satnum(line2, &n2) || n1 != n2) return SGP4_ERR_ARG;

  char buf[32];
  double yy, incl, raan, ecc, argp, ma, mm, bstar;
  if (!field(line1, 19, 20, buf, sizeof buf) || !parse_decimal(buf, &yy)) return SGP4_ERR_ARG;
  if (!field(line1, 21, 32, buf, sizeof buf)) return SGP4_ERR_ARG;
  // day of year: integer part and fraction kept apart (the fraction carries the time)
  const char* dot = std::strchr(buf, '.');
  double frac = 0.0;
  long long iday = 0;
  {
    char ip[16] = {0};
    const size_t ni = dot ? (size_t)(dot - buf) : std::strlen(buf);
    if (ni == 0 || ni >= sizeof ip) return SGP4_ERR_ARG;
    std::memcpy(ip, buf, ni);
    double d;
    if (!parse_decimal(ip, &d) || d < 1.0 || d > 366.0) return SGP4_ERR_ARG;
    iday = (long long)d;
    if (dot) {
      char fp[24] = "0";
      std::strncat(fp, dot, sizeof fp - 2);
      if (!parse_decimal(fp, &frac)) return SGP4_ERR_ARG;
    }
  }
  if (!parse_exp_field(line1, 54, 61, &bstar)) return SGP4_ERR_ARG;
  if (!field(line2, 9, 16, buf, sizeof buf) || !parse_decimal(buf, &incl)) return SGP4_ERR_ARG;
  if (!field(line2, 18, 25, buf, sizeof buf) || !parse_decimal(buf, &raan)) return SGP4_ERR_ARG;
  {
    char eb[48] = "0.";
    if (!field(line2, 27, 33, buf, sizeof buf)) return SGP4_ERR_ARG;
    std::strncat(eb, buf, sizeof eb - 3);
    if (!parse_decimal(eb, &ecc)) return SGP4_ERR_ARG;
  }
  if (!field(line2, 35, 42, buf, sizeof buf) || !parse_decimal(buf, &argp)) return SGP4_ERR_ARG;
  if (!field(line2, 44, 51, buf, sizeof buf) || !parse_decimal(buf, &ma)) return SGP4_ERR_ARG;
  if (!field(line2, 53, 63, buf, sizeof buf) || !parse_decimal(buf, &mm)) return SGP4_ERR_ARG;

  const int y2 = (int)yy;
  if (y2 < 0 || y2 > 99) return SGP4_ERR_ARG;
  const int year = y2 < 57 ? 2000 + y2 : 1900 + y2;
  long long day = jan1(year) + iday - 1;
  double f = 0.5 + frac;
  if (f >= 1.0) { day += 1; f -= 1.0; }

  elements[0] = mm * kRevPerDayToRadPerMin;
  elements[1] = ecc;
  elements[2] = incl * kDeg;
  elements[3] = raan * kDeg;
  elements[4] = argp * kDeg;
  elements[5] = ma * kDeg;
  elements[6] = bstar;
  *epoch_day = (int32_t)day;
  *epoch_frac = f;
  if (satnum) *satnum = n1;
  return SGP4_OK;
}

extern "C" int64_t sgp4_tle_parse_text(const char* text, size_t len, int64_t capacity,
                                       double* elements, int32_t* epoch_day, double* epoch_frac,
                                       int32_t* satnum, int64_t* n_rejected) {
  if (!text || capacity < 0 || (capacity > 0 && (!elements || !epoch_day || !epoch_frac)))
    return -1;
  int64_t n = 0, bad = 0;
  size_t pos = 0;
  char prev[128] = {0};
  bool have_prev = false;
  while (pos < len) {
    size_t end = pos;
    while (end < len && text[end] != '\n') ++end;
    char line[128];
    const size_t m = end - pos < sizeof line - 1 ? end - pos : sizeof line - 1;
    std::memcpy(line, text + pos, m);
    line[m] = '\0';
    pos = end + 1;
    if (line[0] == '2' && have_prev && prev[0] == '1') {
      // Past the capacity the set is still checked and counted, but not stored.
      double el[7], fr;
      int32_t day, num;
      const bool store = n < capacity;
      if (sgp4_tle_parse(prev, line, store ? elements + 7 * n : el, store ? epoch_day + n : &day,
                         store ? epoch_frac + n : &fr, store && satnum ? satnum + n : &num) ==
          SGP4_OK)
        ++n;
      else
        ++bad;
      have_prev = false;
      continue;
    }
    if (line[0] == '1') {
      if (have_prev && prev[0] == '1') ++bad;   // a line 1 without its line 2
      std::memcpy(prev, line, sizeof prev);
      have_prev = true;
    } else {
      if (have_prev && prev[0] == '1') ++bad;
      have_prev = false;                        // a name line (three-line sets) or blank
    }
  }
  if (have_prev && prev[0] == '1') ++bad;
  if (n_rejected) *n_rejected = bad;
  return n;
}

extern "C" sgp4_result sgp4_tle_format(const double* elements, int32_t epoch_day,
                                       double epoch_frac, int32_t satnum, char* line1,
                                       char* line2) {
  if (!elements || !line1 || !line2 || satnum < 0 || satnum > 99999) return SGP4_ERR_ARG;
  if (!(epoch_frac >= 0.0 && epoch_frac < 1.0)) return SGP4_ERR_ARG;
  const double mm = elements[0] / kRevPerDayToRadPerMin;
  const double ecc = elements[1];
  auto deg = [](double rad) {
    double d = std::fmod(rad / kDeg, 360.0);
    return d < 0.0 ? d + 360.0 : d;
  };
  const double incl = elements[2] / kDeg;
  if (!(mm > 0.0 && mm < 100.0) || !(ecc >= 0.0 && ecc < 1.0) || !(incl >= 0.0 && incl <= 180.0))
    return SGP4_ERR_ARG;
  // epoch: year and day of year from the Julian date (0h January 1 is jan1 + 0.5)
  int year = 1957;
  while (year < 2056 && (double)jan1(year + 1) + 0.5 <= (double)epoch_day + epoch_frac) ++year;
  const long long d0 = jan1(year);
  double doy = (double)(epoch_day - d0) + (epoch_frac - 0.5) + 1.0;
  if (doy < 1.0 || doy >= 367.0) return SGP4_ERR_ARG;
  // B*: sign, five-digit mantissa with an implied leading point, exponent digit
  char bs[48];
  {
    const double b = elements[6];
    double a = std::fabs(b);
    int ex = 0;
    long long mant = 0;
    if (a > 0.0) {
      ex = (int)std::floor(std::log10(a)) + 1;
      mant = std::llround(a / std::pow(10.0, ex) * 1e5);
      if (mant >= 100000) { mant /= 10; ex += 1; }
    }
    if (ex < -9 || ex > 9) return SGP4_ERR_ARG;
    std::snprintf(bs, sizeof bs, "%c%05lld%c%d", b < 0.0 ? '-' : ' ', mant, ex < 0 ? '-' : '+',
                  ex < 0 ? -ex : ex);
  }
  char l1[128], l2[128];
  std::snprintf(l1, sizeof l1, "1 %05dU 26001A   %02d%012.8f  .00000000  00000-0 %s 0  999",
                satnum, year % 100, doy, bs);
  std::snprintf(l2, sizeof l2, "2 %05d %8.4f %8.4f %07lld %8.4f %8.4f %11.8f    0", satnum, incl,
                deg(elements[3]), std::llround(ecc * 1e7), deg(elements[4]), deg(elements[5]),
                mm);
  if (std::strlen(l1) != 68 || std::strlen(l2) != 68) return SGP4_ERR_ARG;
  std::memcpy(line1, l1, 68);
  line1[68] = (char)('0' + checksum(l1));
  line1[69] = '\0';
  std::memcpy(line2, l2, 68);
  line2[68] = (char)('0' + checksum(l2));
  line2[69] = '\0';
  return SGP4_OK;
}
