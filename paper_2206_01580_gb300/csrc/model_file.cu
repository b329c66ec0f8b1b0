// Model file: the checkpoint of a trained model (host memory only; no GPU).
//
// A trained model is everything prediction needs (the atomic energy
// partition of the RFF section with the SORF map of the SORF section): the
// FCHL19 parameters, the per-element PCA bases U_e, the SORF signs and phases,
// sigma, the regularisation lambda it was trained with and the weights alpha.
// Layout (little-endian, no padding):
//   "QMLRMDL1"                                       8 bytes
//   u32 version (1), u32 reserved (0)
//   i32 n_el, n2, n3, nfourier; f64 eta2, eta3, N2, N3, c3, zeta, rcut
//   i32 rep_dim, d, n_transform, n_features; f64 sigma, lambda
//   f32 U [n_el][rep_dim][d]
//   u32 sign bits [n_features/d][n_transform][ceil(d/32)] (bit set: -1)
//   f32 b [n_features]
//   f64 alpha [n_features]
//   u64 FNV-1a (64-bit) of every byte before it
// Readers check the magic, the version, the sizes against the file length and
// the checksum before they hand anything out.
#include "common.cuh"

#include <cstdio>
#include <cstring>
#include <vector>

namespace qmlr {

namespace {

constexpr char kMagic[8] = {'Q', 'M', 'L', 'R', 'M', 'D', 'L', '1'};
constexpr uint32_t kVersion = 1;

// Fowler-Noll-Vo FNV-1a, 64-bit: offset basis 14695981039346656037, prime 2^40 + 2^8 + 0xb3.
struct Fnv1a {
  uint64_t h = 14695981039346656037ull;
  void add(const void* p, size_t n) {
    const unsigned char* c = static_cast<const unsigned char*>(p);
    for (size_t i = 0; i < n; ++i) {
      h ^= c[i];
      h *= 1099511628211ull;
    }
  }
};

bool little_endian() {
  const uint32_t one = 1;
  unsigned char c;
  std::memcpy(&c, &one, 1);
  return c == 1;
}

struct Header {
  qmlr_fchl19_params p;
  int32_t rep_dim, d, n_transform, n_features;
  double sigma, lambda;
};

// the fixed part, field by field (no struct padding in the file)
void put_header(std::vector<unsigned char>& out, const Header& h) {
  auto put = [&](const void* v, size_t n) {
    const unsigned char* c = static_cast<const unsigned char*>(v);
    out.insert(out.end(), c, c + n);
  };
  put(kMagic, 8);
  const uint32_t ver = kVersion, res = 0;
  put(&ver, 4);
  put(&res, 4);
  put(&h.p.n_el, 4);
  put(&h.p.n2, 4);
  put(&h.p.n3, 4);
  put(&h.p.nfourier, 4);
  put(&h.p.eta2, 8);
  put(&h.p.eta3, 8);
  put(&h.p.N2, 8);
  put(&h.p.N3, 8);
  put(&h.p.c3, 8);
  put(&h.p.zeta, 8);
  put(&h.p.rcut, 8);
  put(&h.rep_dim, 4);
  put(&h.d, 4);
  put(&h.n_transform, 4);
  put(&h.n_features, 4);
  put(&h.sigma, 8);
  put(&h.lambda, 8);
}

constexpr size_t kHeaderBytes = 8 + 4 + 4 + 4 * 4 + 7 * 8 + 4 * 4 + 2 * 8;

struct Sizes {
  size_t u, bits, b, alpha;
};

// The sizes a model file may hold: exactly what qmlr_model_create accepts
// (FCHL19 parameters in range, rep_dim equal to the one those parameters
// define, d a power of two 16..128, 1..4 transforms, N_F a multiple of d), so
// that a reader never sizes an array from a field the model would disagree with.
bool sizes_of(const Header& h, Sizes* s) {
  if (h.p.n_el < 1 || h.p.n_el > 8 || h.p.n2 < 1 || h.p.n2 > 64 || h.p.n3 < 1 || h.p.n3 > 64 ||
      h.p.nfourier != 1)
    return false;
  if (h.rep_dim != rep_dim_of(h.p)) return false;
  if (!(h.d == 16 || h.d == 32 || h.d == 64 || h.d == 128) || h.n_transform < 1 || h.n_transform > 4 ||
      h.n_features < h.d || h.n_features % h.d != 0)
    return false;
  const size_t words = ((size_t)h.d + 31) / 32;
  s->u = (size_t)h.p.n_el * h.rep_dim * h.d * sizeof(float);
  s->bits = (size_t)(h.n_features / h.d) * h.n_transform * words * sizeof(uint32_t);
  s->b = (size_t)h.n_features * sizeof(float);
  s->alpha = (size_t)h.n_features * sizeof(double);
  return true;
}

// Reads the whole file and checks magic, version, sizes and checksum.
int load(const char* path, Header* h, std::vector<unsigned char>* bytes, Sizes* s) {
  QMLR_REQUIRE(path, "NULL path");
  QMLR_REQUIRE(little_endian(), "model files are little-endian; this host is not");
  FILE* f = std::fopen(path, "rb");
  QMLR_REQUIRE(f, "cannot open model file %s", path);
  std::vector<unsigned char> buf;
  unsigned char chunk[1 << 16];
  size_t got;
  while ((got = std::fread(chunk, 1, sizeof(chunk), f)) > 0) buf.insert(buf.end(), chunk, chunk + got);
  const bool err = std::ferror(f) != 0;
  std::fclose(f);
  QMLR_REQUIRE(!err, "read error on model file %s", path);
  QMLR_REQUIRE(buf.size() >= kHeaderBytes + 8, "model file %s is truncated (%zu bytes)", path, buf.size());
  QMLR_REQUIRE(std::memcmp(buf.data(), kMagic, 8) == 0, "%s is not a model file (bad magic)", path);
  size_t o = 8;
  auto get = [&](void* v, size_t n) {
    std::memcpy(v, buf.data() + o, n);
    o += n;
  };
  uint32_t ver = 0, res = 0;
  get(&ver, 4);
  get(&res, 4);
  QMLR_REQUIRE(ver == kVersion, "model file %s has version %u (this library reads %u)", path, ver, kVersion);
  get(&h->p.n_el, 4);
  get(&h->p.n2, 4);
  get(&h->p.n3, 4);
  get(&h->p.nfourier, 4);
  get(&h->p.eta2, 8);
  get(&h->p.eta3, 8);
  get(&h->p.N2, 8);
  get(&h->p.N3, 8);
  get(&h->p.c3, 8);
  get(&h->p.zeta, 8);
  get(&h->p.rcut, 8);
  get(&h->rep_dim, 4);
  get(&h->d, 4);
  get(&h->n_transform, 4);
  get(&h->n_features, 4);
  get(&h->sigma, 8);
  get(&h->lambda, 8);
  QMLR_REQUIRE(sizes_of(*h, s), "model file %s has inconsistent sizes", path);
  const size_t want = kHeaderBytes + s->u + s->bits + s->b + s->alpha + 8;
  QMLR_REQUIRE(buf.size() == want, "model file %s has %zu bytes, its header implies %zu", path, buf.size(),
               want);
  Fnv1a sum;
  sum.add(buf.data(), want - 8);
  uint64_t stored = 0;
  std::memcpy(&stored, buf.data() + want - 8, 8);
  QMLR_REQUIRE(stored == sum.h, "model file %s fails its checksum", path);
  *bytes = std::move(buf);
  return QMLR_OK;
}

}  // namespace

extern "C" int qmlr_model_file_write(const char* path, const qmlr_fchl19_params* p, int32_t rep_dim, int32_t d,
                                     int32_t n_transform, int32_t n_features, double sigma, double lambda,
                                     const float* host_U, const uint32_t* host_sign_bits, const float* host_b,
                                     const double* host_alpha) {
  QMLR_REQUIRE(path && p && host_U && host_sign_bits && host_b && host_alpha, "NULL pointer argument");
  QMLR_REQUIRE(little_endian(), "model files are little-endian; this host is not");
  Header h{*p, rep_dim, d, n_transform, n_features, sigma, lambda};
  Sizes s{};
  QMLR_REQUIRE(sizes_of(h, &s), "bad model sizes (n_el %d, rep_dim %d, d %d, T %d, N_F %d)", p->n_el, rep_dim,
               d, n_transform, n_features);
  std::vector<unsigned char> out;
  out.reserve(kHeaderBytes + s.u + s.bits + s.b + s.alpha + 8);
  put_header(out, h);
  auto put = [&](const void* v, size_t n) {
    const unsigned char* c = static_cast<const unsigned char*>(v);
    out.insert(out.end(), c, c + n);
  };
  put(host_U, s.u);
  put(host_sign_bits, s.bits);
  put(host_b, s.b);
  put(host_alpha, s.alpha);
  Fnv1a sum;
  sum.add(out.data(), out.size());
  put(&sum.h, 8);
  FILE* f = std::fopen(path, "wb");
  QMLR_REQUIRE(f, "cannot create model file %s", path);
  const size_t wrote = std::fwrite(out.data(), 1, out.size(), f);
  const int closed = std::fclose(f);
  QMLR_REQUIRE(wrote == out.size() && closed == 0, "write error on model file %s", path);
  return QMLR_OK;
}

extern "C" int qmlr_model_file_info(const char* path, qmlr_fchl19_params* p, int32_t* rep_dim, int32_t* d,
                                    int32_t* n_transform, int32_t* n_features, double* sigma, double* lambda) {
  QMLR_REQUIRE(p && rep_dim && d && n_transform && n_features && sigma && lambda, "NULL pointer argument");
  Header h{};
  Sizes s{};
  std::vector<unsigned char> buf;
  const int rc = load(path, &h, &buf, &s);
  if (rc) return rc;
  *p = h.p;
  *rep_dim = h.rep_dim;
  *d = h.d;
  *n_transform = h.n_transform;
  *n_features = h.n_features;
  *sigma = h.sigma;
  *lambda = h.lambda;
  return QMLR_OK;
}

extern "C" int qmlr_model_file_read(const char* path, float* host_U, uint32_t* host_sign_bits, float* host_b,
                                    double* host_alpha) {
  QMLR_REQUIRE(host_U && host_sign_bits && host_b && host_alpha, "NULL pointer argument");
  Header h{};
  Sizes s{};
  std::vector<unsigned char> buf;
  const int rc = load(path, &h, &buf, &s);
  if (rc) return rc;
  size_t o = kHeaderBytes;
  std::memcpy(host_U, buf.data() + o, s.u);
  o += s.u;
  std::memcpy(host_sign_bits, buf.data() + o, s.bits);
  o += s.bits;
  std::memcpy(host_b, buf.data() + o, s.b);
  o += s.b;
  std::memcpy(host_alpha, buf.data() + o, s.alpha);
  return QMLR_OK;
}

}  // namespace qmlr
