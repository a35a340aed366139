// FCIDUMP ingestion (Sec. "Example Usage": the molecular Hamiltonian is read
// from an FCIDUMP file, with a threshold below which integral values are
// neglected).  Host code only.
//
// The format (Knowles and Handy's FCI program): a Fortran namelist header
//   &FCI NORB=N, NELEC=n, MS2=s, ORBSYM=..., ISYM=..., &END   (or "/" to end)
// then one line per integral, "value i j k l" with 1-based orbital indices:
//   i j k l > 0      (ij|kl), standing for its 8 symmetric images;
//   i j > 0, k=l=0   h_ij, standing for h_ji too;
//   i > 0, j=k=l=0   an orbital energy (not part of H; ignored);
//   0 0 0 0          the core energy (a constant added to every energy).
// Fortran exponents ("1.0D-03") are accepted.
#include <cctype>
#include <cerrno>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/cdfci.h"
#include "cdfci_kernels.h"

namespace cdfci {
namespace {

int ffail(int code, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    set_last_error_message(buf);
    return code;
}

// The whole file; false if it cannot be read.
bool slurp(const char *path, std::string &out) {
    FILE *f = fopen(path, "rb");
    if (!f) return false;
    char buf[1 << 16];
    size_t n;
    while ((n = fread(buf, 1, sizeof(buf), f)) > 0) out.append(buf, n);
    const bool ok = !ferror(f);
    fclose(f);
    return ok;
}

// The namelist header [begin, end of "&END" or "/"); body = the first byte after it.
bool split_header(const std::string &s, std::string &hdr, size_t &body) {
    size_t a = 0;
    while (a < s.size() && isspace((unsigned char)s[a])) ++a;
    if (a >= s.size() || s[a] != '&') return false;
    std::string up(s.size() - a, ' ');
    for (size_t i = a; i < s.size(); ++i) up[i - a] = (char)toupper((unsigned char)s[i]);
    size_t e1 = up.find("&END", 4);
    size_t e2 = up.find('/', 4);
    size_t e = std::string::npos, len = 0;
    if (e1 != std::string::npos) { e = e1; len = 4; }
    if (e2 != std::string::npos && (e == std::string::npos || e2 < e)) { e = e2; len = 1; }
    if (e == std::string::npos) return false;
    hdr = up.substr(0, e);
    body = a + e + len;
    return true;
}

// Integer value of KEY= in the header (first occurrence as a whole word); false if absent.
bool header_int(const std::string &hdr, const char *key, long &v) {
    const size_t kl = strlen(key);
    for (size_t p = hdr.find(key); p != std::string::npos; p = hdr.find(key, p + 1)) {
        const bool start = p == 0 || !(isalnum((unsigned char)hdr[p - 1]) || hdr[p - 1] == '_');
        size_t q = p + kl;
        while (q < hdr.size() && isspace((unsigned char)hdr[q])) ++q;
        if (!start || q >= hdr.size() || hdr[q] != '=') continue;
        ++q;
        while (q < hdr.size() && isspace((unsigned char)hdr[q])) ++q;
        char *endp = nullptr;
        errno = 0;
        const long x = strtol(hdr.c_str() + q, &endp, 10);
        if (endp == hdr.c_str() + q || errno) return false;
        v = x;
        return true;
    }
    return false;
}

int parse_header(const std::string &s, int *norb, int *nelec, int *ms2, size_t *body) {
    std::string hdr;
    size_t b = 0;
    if (!split_header(s, hdr, b)) return ffail(CDFCI_ERR_ARG, "FCIDUMP: no &FCI ... &END (or /) header");
    long N = 0, ne = 0, m2 = 0;
    if (!header_int(hdr, "NORB", N) || !header_int(hdr, "NELEC", ne))
        return ffail(CDFCI_ERR_ARG, "FCIDUMP: header lacks NORB or NELEC");
    if (!header_int(hdr, "MS2", m2)) m2 = 0;
    if (N < 1 || N > 63) return ffail(CDFCI_ERR_ARG, "FCIDUMP: NORB = %ld outside [1, 63]", N);
    if (ne < 0 || ne > 2 * N || m2 < -ne || m2 > ne || ((ne + m2) & 1))
        return ffail(CDFCI_ERR_ARG, "FCIDUMP: NELEC = %ld, MS2 = %ld inconsistent with NORB = %ld", ne, m2, N);
    if ((ne + m2) / 2 > N || (ne - m2) / 2 > N)
        return ffail(CDFCI_ERR_ARG, "FCIDUMP: more electrons of one spin than orbitals");
    *norb = (int)N;
    *nelec = (int)ne;
    *ms2 = (int)m2;
    if (body) *body = b;
    return CDFCI_OK;
}

// One number (Fortran D exponents accepted); advances p.  False at the end of the line or on junk.
bool next_number(const char *&p, const char *end, double &x) {
    while (p < end && (*p == ' ' || *p == '\t' || *p == ',' || *p == '\r')) ++p;
    if (p >= end || *p == '\n') return false;
    char tok[64];
    int n = 0;
    while (p < end && !isspace((unsigned char)*p) && *p != ',' && n < 63) {
        tok[n++] = (*p == 'D' || *p == 'd') ? 'E' : *p;
        ++p;
    }
    tok[n] = 0;
    char *endp = nullptr;
    x = strtod(tok, &endp);
    return endp != tok && *endp == 0;
}

}  // namespace
}  // namespace cdfci

using namespace cdfci;

extern "C" __attribute__((visibility("default"))) int cdfci_fcidump_header(const char *path, int *norb, int *nelec,
                                                                          int *ms2) {
    if (!path || !norb || !nelec || !ms2) return ffail(CDFCI_ERR_ARG, "cdfci_fcidump_header: NULL argument");
    std::string s;
    if (!slurp(path, s)) return ffail(CDFCI_ERR_ARG, "FCIDUMP: cannot read %s", path);
    return parse_header(s, norb, nelec, ms2, nullptr);
}

extern "C" __attribute__((visibility("default"))) int cdfci_fcidump_read(const char *path, double threshold, int norb,
                                                                        double *h, double *g, double *e_core) {
    if (!path || !h || !g) return ffail(CDFCI_ERR_ARG, "cdfci_fcidump_read: NULL argument");
    if (!(threshold >= 0.0) || !std::isfinite(threshold))
        return ffail(CDFCI_ERR_ARG, "cdfci_fcidump_read: threshold must be finite and >= 0");
    std::string s;
    if (!slurp(path, s)) return ffail(CDFCI_ERR_ARG, "FCIDUMP: cannot read %s", path);
    int N = 0, ne = 0, m2 = 0;
    size_t body = 0;
    const int rc = parse_header(s, &N, &ne, &m2, &body);
    if (rc) return rc;
    if (N != norb) return ffail(CDFCI_ERR_ARG, "cdfci_fcidump_read: file has NORB = %d, caller gave %d", N, norb);
    const size_t n2 = (size_t)N * N, n4 = n2 * n2;
    std::vector<double> hv(n2, 0.0), gv(n4, 0.0);
    double core = 0.0;
    const char *p = s.c_str() + body, *end = s.c_str() + s.size();
    long line = 0;
    while (p < end) {
        // one line: value i j k l
        ++line;
        const char *eol = (const char *)memchr(p, '\n', (size_t)(end - p));
        if (!eol) eol = end;
        const char *q = p;
        double x = 0.0, fi = 0.0, fj = 0.0, fk = 0.0, fl = 0.0;
        bool any = false;
        {
            const char *t = q;
            while (t < eol && isspace((unsigned char)*t)) ++t;
            any = t < eol;
        }
        if (any) {
            if (!next_number(q, eol, x) || !next_number(q, eol, fi) || !next_number(q, eol, fj) ||
                !next_number(q, eol, fk) || !next_number(q, eol, fl))
                return ffail(CDFCI_ERR_ARG, "FCIDUMP: integral line %ld is not 'value i j k l'", line);
            const int i = (int)fi, j = (int)fj, k = (int)fk, l = (int)fl;
            if (fi != i || fj != j || fk != k || fl != l || i < 0 || j < 0 || k < 0 || l < 0 || i > N || j > N ||
                k > N || l > N)
                return ffail(CDFCI_ERR_ARG, "FCIDUMP: integral line %ld has indices outside [0, %d]", line, N);
            if (!std::isfinite(x)) return ffail(CDFCI_ERR_NONFINITE, "FCIDUMP: integral line %ld is not finite", line);
            const double v = fabs(x) < threshold ? 0.0 : x;
            if (i > 0 && j > 0 && k > 0 && l > 0) {
                const size_t a = i - 1, b = j - 1, c = k - 1, d = l - 1;
                const size_t idx[8][4] = {{a, b, c, d}, {b, a, c, d}, {a, b, d, c}, {b, a, d, c},
                                          {c, d, a, b}, {d, c, a, b}, {c, d, b, a}, {d, c, b, a}};
                for (const auto &t : idx) gv[((t[0] * N + t[1]) * N + t[2]) * N + t[3]] = v;
            } else if (i > 0 && j > 0 && k == 0 && l == 0) {
                hv[(size_t)(i - 1) * N + (j - 1)] = v;
                hv[(size_t)(j - 1) * N + (i - 1)] = v;
            } else if (i == 0 && j == 0 && k == 0 && l == 0) {
                core = x;                        // a constant: never truncated
            } else if (!(i > 0 && j == 0 && k == 0 && l == 0)) {
                return ffail(CDFCI_ERR_ARG, "FCIDUMP: integral line %ld has index pattern %d %d %d %d", line, i, j, k,
                             l);
            }
        }
        p = eol < end ? eol + 1 : end;
    }
    memcpy(h, hv.data(), n2 * sizeof(double));
    memcpy(g, gv.data(), n4 * sizeof(double));
    if (e_core) *e_core = core;
    return CDFCI_OK;
}
