// The .qtt operator file: a fixed header, the ranks, then the FP64 cores in
// the layout qtt_create takes, so that every consumer (the library, the
// generators, the oracle) reads identical bits.  Host code only; no
// counterpart in the paper (it stores cores in Matlab cells).
//
// Layout, all little-endian:
//   bytes  0-3   magic "QTT1"
//   4-7          format version (1)
//   8-11         d (1..30)
//   12-15        element type (0 = FP64)
//   16-19        core layout (0 = C-order [r_k][i][j][r_{k+1}], i the row bit)
//   20-23        reserved (0)
//   24 ..        d + 1 ranks (uint32), then sum_k 4 r_k r_{k+1} FP64 values
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "qtt_internal.h"

namespace qtt {
namespace {

constexpr char kMagic[4] = {'Q', 'T', 'T', '1'};
constexpr uint32_t kVersion = 1;

void put_u32(unsigned char *p, uint32_t v) {
  for (int b = 0; b < 4; ++b) p[b] = (unsigned char)((v >> (8 * b)) & 0xFFu);
}
uint32_t get_u32(const unsigned char *p) {
  return (uint32_t)p[0] | ((uint32_t)p[1] << 8) | ((uint32_t)p[2] << 16) | ((uint32_t)p[3] << 24);
}
void put_f64(unsigned char *p, double v) {
  uint64_t u;
  std::memcpy(&u, &v, 8);
  for (int b = 0; b < 8; ++b) p[b] = (unsigned char)((u >> (8 * b)) & 0xFFu);
}
double get_f64(const unsigned char *p) {
  uint64_t u = 0;
  for (int b = 0; b < 8; ++b) u |= (uint64_t)p[b] << (8 * b);
  double v;
  std::memcpy(&v, &u, 8);
  return v;
}

// ranks valid for an operator: d in 1..30, ends 1, 1 <= r <= 4096
bool ranks_ok(int d, const int *ranks) {
  if (d < 1 || d > 30 || !ranks || ranks[0] != 1 || ranks[d] != 1) return false;
  for (int k = 0; k <= d; ++k)
    if (ranks[k] < 1 || ranks[k] > 4096) return false;
  return true;
}
int64_t core_len(int d, const int *ranks) {
  int64_t n = 0;
  for (int k = 0; k < d; ++k) n += (int64_t)4 * ranks[k] * ranks[k + 1];
  return n;
}

}  // namespace
}  // namespace qtt

using namespace qtt;

extern "C" {

qtt_status qtt_write_file(const char *path, int d, const int *ranks, const double *cores) {
  if (!path || !cores || !ranks_ok(d, ranks))
    return fail(QTT_ERR_INVALID_ARG, "qtt_write_file: bad path, d, ranks or cores");
  const int64_t n = core_len(d, ranks);
  std::vector<unsigned char> buf((size_t)(24 + 4 * (d + 1)) + (size_t)n * 8);
  std::memcpy(buf.data(), kMagic, 4);
  put_u32(&buf[4], kVersion);
  put_u32(&buf[8], (uint32_t)d);
  put_u32(&buf[12], 0);
  put_u32(&buf[16], 0);
  put_u32(&buf[20], 0);
  for (int k = 0; k <= d; ++k) put_u32(&buf[24 + 4 * k], (uint32_t)ranks[k]);
  unsigned char *c = &buf[24 + 4 * (d + 1)];
  for (int64_t e = 0; e < n; ++e) put_f64(c + 8 * e, cores[e]);
  FILE *f = std::fopen(path, "wb");
  if (!f) return fail(QTT_ERR_INVALID_ARG, std::string("qtt_write_file: cannot open ") + path);
  const size_t w = std::fwrite(buf.data(), 1, buf.size(), f);
  const int cl = std::fclose(f);
  if (w != buf.size() || cl != 0)
    return fail(QTT_ERR_INVALID_ARG, std::string("qtt_write_file: write failed: ") + path);
  return QTT_OK;
}

qtt_status qtt_read_file(const char *path, int *d, int *ranks, int ranks_cap, double *cores,
                         int64_t cores_cap, int64_t *cores_len) {
  if (!path || !d) return fail(QTT_ERR_INVALID_ARG, "qtt_read_file: bad path or d");
  FILE *f = std::fopen(path, "rb");
  if (!f) return fail(QTT_ERR_INVALID_ARG, std::string("qtt_read_file: cannot open ") + path);
  std::vector<unsigned char> buf;
  unsigned char tmp[65536];
  size_t got;
  while ((got = std::fread(tmp, 1, sizeof(tmp), f)) > 0) buf.insert(buf.end(), tmp, tmp + got);
  std::fclose(f);
  if (buf.size() < 24 || std::memcmp(buf.data(), kMagic, 4) != 0)
    return fail(QTT_ERR_INVALID_ARG, "qtt_read_file: not a .qtt file (magic)");
  if (get_u32(&buf[4]) != kVersion)
    return fail(QTT_ERR_UNSUPPORTED, "qtt_read_file: unsupported format version");
  if (get_u32(&buf[12]) != 0 || get_u32(&buf[16]) != 0)
    return fail(QTT_ERR_UNSUPPORTED, "qtt_read_file: unsupported element type or layout");
  const uint32_t dd = get_u32(&buf[8]);
  if (dd < 1 || dd > 30 || buf.size() < 24 + 4 * ((size_t)dd + 1))
    return fail(QTT_ERR_INVALID_ARG, "qtt_read_file: bad d or truncated header");
  std::vector<int> r(dd + 1);
  for (uint32_t k = 0; k <= dd; ++k) r[k] = (int)get_u32(&buf[24 + 4 * k]);
  if (!ranks_ok((int)dd, r.data())) return fail(QTT_ERR_INVALID_ARG, "qtt_read_file: bad ranks");
  const int64_t n = core_len((int)dd, r.data());
  const size_t want = 24 + 4 * ((size_t)dd + 1) + (size_t)n * 8;
  if (buf.size() != want)
    return fail(QTT_ERR_INVALID_ARG, "qtt_read_file: file length does not match the ranks");
  *d = (int)dd;
  if (cores_len) *cores_len = n;
  if (ranks) {
    if (ranks_cap < (int)dd + 1) return fail(QTT_ERR_INVALID_ARG, "qtt_read_file: ranks_cap < d + 1");
    for (uint32_t k = 0; k <= dd; ++k) ranks[k] = r[k];
  }
  if (cores) {
    if (cores_cap < n) return fail(QTT_ERR_INVALID_ARG, "qtt_read_file: cores_cap too small");
    const unsigned char *c = &buf[24 + 4 * (dd + 1)];
    for (int64_t e = 0; e < n; ++e) cores[e] = get_f64(c + 8 * e);
  }
  return QTT_OK;
}

}  // extern "C"
