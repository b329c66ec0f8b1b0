// Periodic environments: for every atom i of a periodic system, the lattice
// images R_j + n . cell (n an integer triple; every atom j, i's own images
// included, i itself excluded) closer than r_cut to R_i -- the neighbourhood
// the FCHL19 sums run over for the paper's periodic MOF and water systems.
// Host code (a setup step per configuration): a cell list in fractional
// coordinates. The cell is cut into n_a bins along lattice vector a, with
// n_a = max(1, floor(h_a / r_cut)) and h_a the spacing of the lattice planes
// normal to the other two vectors, so a bin is at least r_cut thick; an atom's
// search then spans ceil(r_cut n_a / h_a) bins either way along each axis
// (one when the cell is large, several when r_cut exceeds the cell), each bin
// offset naming one (bin, lattice translation) pair, so no image is visited
// twice. The translation is reported relative to the caller's coordinates
// (atoms outside [0, 1) in fractional coordinates are wrapped for binning
// only). Entries of one atom are sorted by (j, n).
#include "common.cuh"

#include <algorithm>
#include <cmath>
#include <vector>

namespace qmlr {

namespace {

struct Env {
  int32_t j, n0, n1, n2;
  bool operator<(const Env& o) const {
    if (j != o.j) return j < o.j;
    if (n0 != o.n0) return n0 < o.n0;
    if (n1 != o.n1) return n1 < o.n1;
    return n2 < o.n2;
  }
};

struct Cells {
  double A[3][3];      // lattice vectors as rows
  double Ainv[3][3];   // inverse (fractional = cartesian x Ainv)
  int nb[3];           // bins per axis
  int reach[3];        // bin offsets searched either way
};

bool setup(const double* cell, double rcut, Cells* c) {
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) c->A[a][b] = cell[3 * a + b];
  const double(&A)[3][3] = c->A;
  const double det = A[0][0] * (A[1][1] * A[2][2] - A[1][2] * A[2][1]) -
                     A[0][1] * (A[1][0] * A[2][2] - A[1][2] * A[2][0]) +
                     A[0][2] * (A[1][0] * A[2][1] - A[1][1] * A[2][0]);
  if (!(std::fabs(det) > 0) || !std::isfinite(det)) return false;
  // inverse by cofactors: Ainv[b][a] = cof(a, b) / det
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      const int a1 = (a + 1) % 3, a2 = (a + 2) % 3, b1 = (b + 1) % 3, b2 = (b + 2) % 3;
      c->Ainv[b][a] = (A[a1][b1] * A[a2][b2] - A[a1][b2] * A[a2][b1]) / det;
    }
  for (int a = 0; a < 3; ++a) {
    const double* u = A[(a + 1) % 3];
    const double* w = A[(a + 2) % 3];
    const double cx = u[1] * w[2] - u[2] * w[1], cy = u[2] * w[0] - u[0] * w[2], cz = u[0] * w[1] - u[1] * w[0];
    const double h = std::fabs(det) / std::sqrt(cx * cx + cy * cy + cz * cz);
    c->nb[a] = std::max(1, (int)std::floor(h / rcut));
    c->reach[a] = (int)std::ceil(rcut * c->nb[a] / h);
  }
  return true;
}

// environments of every atom, each sorted by (j, n)
int build(const double* x, int n_atoms, const double* cell, double rcut, std::vector<std::vector<Env>>* env) {
  Cells c;
  QMLR_REQUIRE(setup(cell, rcut, &c), "the cell is singular or not finite");
  const long nbins = (long)c.nb[0] * c.nb[1] * c.nb[2];
  QMLR_REQUIRE(nbins <= (1L << 24), "too many cell-list bins (%ld)", nbins);
  std::vector<int> bin(n_atoms), wrap(3 * (size_t)n_atoms);
  std::vector<int> cnt(nbins + 1, 0);
  for (int i = 0; i < n_atoms; ++i) {
    int b3[3];
    for (int a = 0; a < 3; ++a) {
      const double s = x[3 * i] * c.Ainv[0][a] + x[3 * i + 1] * c.Ainv[1][a] + x[3 * i + 2] * c.Ainv[2][a];
      QMLR_REQUIRE(std::isfinite(s), "atom %d has a non-finite coordinate", i);
      const double fl = std::floor(s);
      wrap[3 * i + a] = (int)fl;   // s - fl in [0, 1)
      b3[a] = std::min(c.nb[a] - 1, (int)((s - fl) * c.nb[a]));
    }
    bin[i] = (b3[0] * c.nb[1] + b3[1]) * c.nb[2] + b3[2];
    ++cnt[bin[i] + 1];
  }
  for (long b = 0; b < nbins; ++b) cnt[b + 1] += cnt[b];
  std::vector<int> members(n_atoms), fill(cnt.begin(), cnt.end() - 1);
  for (int i = 0; i < n_atoms; ++i) members[fill[bin[i]]++] = i;
  const double rc2 = rcut * rcut;
  env->assign(n_atoms, {});
  for (int i = 0; i < n_atoms; ++i) {
    const int bi0 = bin[i] / (c.nb[1] * c.nb[2]), bi1 = (bin[i] / c.nb[2]) % c.nb[1], bi2 = bin[i] % c.nb[2];
    std::vector<Env>& e = (*env)[i];
    for (int d0 = -c.reach[0]; d0 <= c.reach[0]; ++d0)
      for (int d1 = -c.reach[1]; d1 <= c.reach[1]; ++d1)
        for (int d2 = -c.reach[2]; d2 <= c.reach[2]; ++d2) {
          const int t[3] = {bi0 + d0, bi1 + d1, bi2 + d2};
          int bb[3], tr[3];
          for (int a = 0; a < 3; ++a) {
            bb[a] = ((t[a] % c.nb[a]) + c.nb[a]) % c.nb[a];
            tr[a] = (t[a] - bb[a]) / c.nb[a];   // exact: t - bb is a multiple of nb
          }
          const long b = ((long)bb[0] * c.nb[1] + bb[1]) * c.nb[2] + bb[2];
          for (int m = cnt[b]; m < cnt[b + 1]; ++m) {
            const int j = members[m];
            // translation relative to the caller's coordinates
            const int n0 = tr[0] + wrap[3 * i] - wrap[3 * j];
            const int n1 = tr[1] + wrap[3 * i + 1] - wrap[3 * j + 1];
            const int n2 = tr[2] + wrap[3 * i + 2] - wrap[3 * j + 2];
            if (j == i && n0 == 0 && n1 == 0 && n2 == 0) continue;
            double v2 = 0;
            for (int k = 0; k < 3; ++k) {
              const double v = x[3 * j + k] + n0 * c.A[0][k] + n1 * c.A[1][k] + n2 * c.A[2][k] - x[3 * i + k];
              v2 += v * v;
            }
            if (v2 < rc2) e.push_back({j, n0, n1, n2});
          }
        }
    std::sort(e.begin(), e.end());
  }
  return QMLR_OK;
}

int check_args(const double* x, int32_t n_atoms, const double* cell, double rcut) {
  QMLR_REQUIRE(n_atoms >= 0 && (n_atoms == 0 || x) && cell, "bad arguments");
  QMLR_REQUIRE(rcut > 0 && std::isfinite(rcut), "r_cut must be positive and finite");
  return QMLR_OK;
}

}  // namespace

extern "C" int qmlr_periodic_environment_count(const double* host_coords, int32_t n_atoms, const double* host_cell,
                                               double rcut, int64_t* host_env_ptr) {
  if (int rc = check_args(host_coords, n_atoms, host_cell, rcut)) return rc;
  QMLR_REQUIRE(host_env_ptr, "NULL env_ptr");
  std::vector<std::vector<Env>> env;
  if (int rc = build(host_coords, n_atoms, host_cell, rcut, &env)) return rc;
  host_env_ptr[0] = 0;
  for (int i = 0; i < n_atoms; ++i) host_env_ptr[i + 1] = host_env_ptr[i] + (int64_t)env[i].size();
  return QMLR_OK;
}

extern "C" int qmlr_periodic_environment(const double* host_coords, int32_t n_atoms, const double* host_cell,
                                         double rcut, const int64_t* host_env_ptr, int32_t* host_env_atom,
                                         int32_t* host_env_shift) {
  if (int rc = check_args(host_coords, n_atoms, host_cell, rcut)) return rc;
  QMLR_REQUIRE(host_env_ptr && (host_env_ptr[n_atoms] == 0 || (host_env_atom && host_env_shift)),
               "NULL output");
  std::vector<std::vector<Env>> env;
  if (int rc = build(host_coords, n_atoms, host_cell, rcut, &env)) return rc;
  for (int i = 0; i < n_atoms; ++i) {
    QMLR_REQUIRE(host_env_ptr[i + 1] - host_env_ptr[i] == (int64_t)env[i].size(),
                 "env_ptr does not match these coordinates (atom %d)", i);
    int64_t o = host_env_ptr[i];
    for (const Env& e : env[i]) {
      host_env_atom[o] = e.j;
      host_env_shift[3 * o] = e.n0;
      host_env_shift[3 * o + 1] = e.n1;
      host_env_shift[3 * o + 2] = e.n2;
      ++o;
    }
  }
  return QMLR_OK;
}

}  // namespace qmlr

extern "C" int qmlr_periodic_reverse(const int64_t* host_env_ptr, const int32_t* host_env_atom, int32_t n_atoms,
                                     int64_t* host_rev_ptr, int64_t* host_rev_entry) {
  QMLR_REQUIRE(n_atoms >= 0, "n_atoms must be >= 0");
  QMLR_REQUIRE(host_env_ptr && host_rev_ptr, "NULL pointer argument");
  const int64_t E = host_env_ptr[n_atoms];
  QMLR_REQUIRE(E >= 0 && (E == 0 || (host_env_atom && host_rev_entry)), "NULL pointer argument");
  std::vector<int64_t> cnt((size_t)n_atoms + 1, 0);
  for (int64_t e = 0; e < E; ++e) {
    const int32_t j = host_env_atom[e];
    QMLR_REQUIRE(j >= 0 && j < n_atoms, "env_atom[%lld] = %d out of range", (long long)e, j);
    ++cnt[(size_t)j + 1];
  }
  host_rev_ptr[0] = 0;
  for (int k = 0; k < n_atoms; ++k) host_rev_ptr[k + 1] = host_rev_ptr[k] + cnt[(size_t)k + 1];
  std::vector<int64_t> pos(host_rev_ptr, host_rev_ptr + n_atoms);
  for (int64_t e = 0; e < E; ++e) host_rev_entry[pos[(size_t)host_env_atom[e]]++] = e;
  return QMLR_OK;
}
