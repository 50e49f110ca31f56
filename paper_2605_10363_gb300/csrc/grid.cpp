// kldi_make_grid: atom-centred molecular grid (App. A "Numerical integration
// grids"), Becke partition, per-atom Morton order (App. B Eq. morton_code) and
// 128-point blocks.  Host C++ with OpenMP: this is geometry-fixed
// preprocessing, run once per geometry (Sec. III-D); the Becke weights run on
// the GPU when one is present (grid_dev.cu), else on the host cores.
//
// Radial: Treutler-Ahlrichs M4 map r = (xi/ln2)(1+x)^0.6 ln(2/(1-x)), xi = 1, on
// Chebyshev second-kind nodes x_i = cos(i pi/(n+1)) with weights
// pi/(n+1) sin(i pi/(n+1)) for int_{-1}^{1}; shells listed by increasing r.
// Angular: Gauss-Legendre in cos(theta) (n_theta nodes, ascending) times
// 2 n_theta azimuths 2 pi k / (2 n_theta); theta-major order.
// Becke: three iterations of p(mu) = 1.5 mu - 0.5 mu^3, no size adjustment.
// Factors of a cell function are multiplied nearest atom first and a cell
// value is dropped once it falls below 1e-40 (an absolute change of at most
// natm * 1e-40 in the normaliser).
#include <omp.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdint>
#include <cstring>
#include <memory>
#include <numeric>

#include "internal.h"

namespace kldi {

static thread_local std::string g_err;

void set_error(const char* fmt, ...) {
  char buf[1024];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_err = buf;
}

const char* last_error() { return g_err.c_str(); }

static void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w) {
  // Newton iteration on the three-term recurrence of P_n; nodes ascending.
  x.assign(n, 0.0);
  w.assign(n, 0.0);
  for (int i = 0; i < n; ++i) {
    double z = std::cos(M_PI * (i + 0.75) / (n + 0.5));
    double dp = 0.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= n; ++k) {
        const double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      if (n == 1) { p0 = 1.0; p1 = z; }
      dp = n * (z * p1 - p0) / (z * z - 1.0);
      const double dz = p1 / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) {
        double q0 = 1.0, q1 = z;
        for (int k = 2; k <= n; ++k) {
          const double q2 = ((2.0 * k - 1.0) * z * q1 - (k - 1.0) * q0) / k;
          q0 = q1;
          q1 = q2;
        }
        dp = n * (z * q1 - q0) / (z * z - 1.0);
        break;
      }
    }
    x[n - 1 - i] = z;  // cos of increasing angle decreases: store ascending
    w[n - 1 - i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

static inline double becke_s(double mu) {
  double p = mu;
  for (int k = 0; k < 3; ++k) p = 1.5 * p - 0.5 * p * p * p;
  return 0.5 * (1.0 - p);
}

static inline uint64_t morton60(uint64_t x, uint64_t y, uint64_t z) {
  uint64_t m = 0;
  for (int k = 0; k < 20; ++k) {
    m |= ((z >> k) & 1ull) << (3 * k);
    m |= ((y >> k) & 1ull) << (3 * k + 1);
    m |= ((x >> k) & 1ull) << (3 * k + 2);
  }
  return m;
}

}  // namespace kldi

extern "C" const char* kldi_last_error(void) { return kldi::last_error(); }

extern "C" kldi_status kldi_make_grid(const kldi_molecule* mol, const kldi_grid_spec* spec, kldi_grid** out) {
  return kldi::guarded("kldi_make_grid", [&]() -> kldi_status {
    using namespace kldi;
    if (!mol || !spec || !out || mol->natm <= 0 || !mol->xyz || !mol->Z) {
      set_error("kldi_make_grid: null argument or natm <= 0");
      return KLDI_EINVAL;
    }
    for (int64_t k = 0; k < 3 * (int64_t)mol->natm; ++k)
      if (!std::isfinite(mol->xyz[k])) {
        set_error("kldi_make_grid: atom %lld has a non-finite coordinate", (long long)(k / 3));
        return KLDI_EINVAL;
      }
    if (spec->nrad <= 0 || spec->nregions <= 0 || !spec->ntheta) {
      set_error("kldi_make_grid: bad grid spec");
      return KLDI_EINVAL;
    }
    if (spec->block != kBlockPts) {
      set_error("kldi_make_grid: only block = %d is supported", kBlockPts);
      return KLDI_EUNSUPPORTED;
    }
    for (int r = 0; r < spec->nregions; ++r)
      if (spec->ntheta[r] <= 0 || spec->ntheta[r] > 128) {
        set_error("kldi_make_grid: ntheta out of range");
        return KLDI_EINVAL;
      }
    const int natm = mol->natm;
    const int nrad = spec->nrad;
    // radial rule, increasing r
    std::vector<double> rr(nrad), wr(nrad);
    for (int i = 1; i <= nrad; ++i) {
      const double th = i * M_PI / (nrad + 1);
      const double x = std::cos(th);
      const double wx = M_PI / (nrad + 1) * std::sin(th);
      const double l2 = std::log(2.0);
      const double r = 1.0 / l2 * std::pow(1.0 + x, 0.6) * std::log(2.0 / (1.0 - x));
      const double dr = 1.0 / l2 * (0.6 * std::pow(1.0 + x, 0.6 - 1.0) * std::log(2.0 / (1.0 - x)) +
                                    std::pow(1.0 + x, 0.6) / (1.0 - x));
      rr[nrad - i] = r;
      wr[nrad - i] = wx * dr * r * r;
    }
    // angular rules per region
    struct Ang { std::vector<double> dx, dy, dz, w; };
    std::vector<Ang> ang(spec->nregions);
    for (int reg = 0; reg < spec->nregions; ++reg) {
      const int nt = spec->ntheta[reg], np = 2 * nt;
      std::vector<double> t, wt;
      gauss_legendre(nt, t, wt);
      Ang& a = ang[reg];
      for (int j = 0; j < nt; ++j) {
        const double st = std::sqrt(1.0 - t[j] * t[j]);
        for (int k = 0; k < np; ++k) {
          const double phi = 2.0 * M_PI * k / np;
          a.dx.push_back(st * std::cos(phi));
          a.dy.push_back(st * std::sin(phi));
          a.dz.push_back(t[j]);
          a.w.push_back(wt[j] * (2.0 * M_PI / np));
        }
      }
    }
    int64_t per_atom = 0;
    for (int ir = 0; ir < nrad; ++ir) {
      const int reg = std::min(ir * spec->nregions / nrad, spec->nregions - 1);
      per_atom += (int64_t)ang[reg].w.size();
    }
    const int64_t nreal = per_atom * natm;
    const int64_t npoints = (nreal + kBlockPts - 1) / kBlockPts * kBlockPts;
    kldi_grid* G = new (std::nothrow) kldi_grid;
    if (!G) { set_error("kldi_make_grid: out of host memory"); return KLDI_ENOMEM; }
    G->npoints = npoints;
    G->nreal = nreal;
    G->nblocks = npoints / kBlockPts;
    G->xyz.resize(npoints * 3);
    G->w.resize(npoints);
    G->atom.resize(npoints);
    std::vector<double> raw_w(npoints, 0.0);
    const double* A = mol->xyz;

    // points per atom, Morton-sorted within the atom
  #pragma omp parallel for schedule(dynamic)
    for (int a = 0; a < natm; ++a) {
      std::vector<double> px, py, pz, pw;
      px.reserve(per_atom); py.reserve(per_atom); pz.reserve(per_atom); pw.reserve(per_atom);
      for (int ir = 0; ir < nrad; ++ir) {
        const int reg = std::min(ir * spec->nregions / nrad, spec->nregions - 1);
        const Ang& an = ang[reg];
        for (size_t k = 0; k < an.w.size(); ++k) {
          px.push_back(A[3 * a + 0] + rr[ir] * an.dx[k]);
          py.push_back(A[3 * a + 1] + rr[ir] * an.dy[k]);
          pz.push_back(A[3 * a + 2] + rr[ir] * an.dz[k]);
          pw.push_back(wr[ir] * an.w[k]);
        }
      }
      const double lx = *std::min_element(px.begin(), px.end());
      const double ly = *std::min_element(py.begin(), py.end());
      const double lz = *std::min_element(pz.begin(), pz.end());
      const int64_t n = (int64_t)px.size();
      std::vector<uint64_t> key(n);
      auto lat = [](double v) -> uint64_t {
        double q = std::floor(v * 128.0);
        if (q < 0) q = 0;
        if (q > 1048575.0) q = 1048575.0;
        return (uint64_t)q;
      };
      for (int64_t k = 0; k < n; ++k) key[k] = morton60(lat(px[k] - lx), lat(py[k] - ly), lat(pz[k] - lz));
      std::vector<int64_t> ord(n);
      std::iota(ord.begin(), ord.end(), 0);
      std::stable_sort(ord.begin(), ord.end(), [&](int64_t i, int64_t j) { return key[i] < key[j]; });
      const int64_t base = (int64_t)a * per_atom;
      for (int64_t k = 0; k < n; ++k) {
        const int64_t s = ord[k];
        G->xyz[(base + k) * 3 + 0] = px[s];
        G->xyz[(base + k) * 3 + 1] = py[s];
        G->xyz[(base + k) * 3 + 2] = pz[s];
        raw_w[base + k] = pw[s];
        G->atom[base + k] = a;
      }
    }
    for (int64_t k = nreal; k < npoints; ++k) {
      for (int c = 0; c < 3; ++c) G->xyz[k * 3 + c] = G->xyz[(nreal - 1) * 3 + c];
      G->atom[k] = G->atom[nreal - 1];
    }

    // Becke weights
    std::vector<double> R(natm * (int64_t)natm);
    for (int b = 0; b < natm; ++b)
      for (int c = 0; c < natm; ++c) {
        const double dx = A[3 * b] - A[3 * c], dy = A[3 * b + 1] - A[3 * c + 1], dz = A[3 * b + 2] - A[3 * c + 2];
        R[(int64_t)b * natm + c] = std::sqrt(dx * dx + dy * dy + dz * dz);
      }
    // neighbour order of every atom (by distance), used as the multiplication order
    std::vector<int32_t> nbr(natm * (int64_t)natm);
    for (int a = 0; a < natm; ++a) {
      int32_t* o = &nbr[(int64_t)a * natm];
      std::iota(o, o + natm, 0);
      std::stable_sort(o, o + natm, [&](int32_t i, int32_t j) { return R[(int64_t)a * natm + i] < R[(int64_t)a * natm + j]; });
    }
    // on the current CUDA device when there is one (same arithmetic), else on the host cores
    int ndev = 0;
    const bool use_dev = natm > 1 && cudaGetDeviceCount(&ndev) == cudaSuccess && ndev > 0;
    cudaGetLastError();
    if (use_dev) {
      const kldi_status st = becke_weights_device(natm, A, R.data(), nbr.data(), G->xyz.data(), G->atom.data(),
                                                  raw_w.data(), nreal, G->w.data());
      if (st != KLDI_OK) {
        delete G;
        return st;
      }
    } else
  #pragma omp parallel
    {
      std::vector<double> d(natm);
  #pragma omp for schedule(dynamic, 256)
      for (int64_t k = 0; k < nreal; ++k) {
        if (natm == 1) { G->w[k] = raw_w[k]; continue; }
        const double x = G->xyz[k * 3], y = G->xyz[k * 3 + 1], z = G->xyz[k * 3 + 2];
        const int own = G->atom[k];
        for (int b = 0; b < natm; ++b) {
          const double dx = x - A[3 * b], dy = y - A[3 * b + 1], dz = z - A[3 * b + 2];
          d[b] = std::sqrt(dx * dx + dy * dy + dz * dz);
        }
        const int32_t* order = &nbr[(int64_t)own * natm];
        double sum = 0.0, pown = 0.0;
        for (int ib = 0; ib < natm; ++ib) {
          const int b = order[ib];
          double P = 1.0;
          for (int ic = 0; ic < natm; ++ic) {
            const int c = order[ic];
            if (c == b) continue;
            P *= becke_s((d[b] - d[c]) / R[(int64_t)b * natm + c]);
            if (P < 1e-40) { P = 0.0; break; }
          }
          sum += P;
          if (b == own) pown = P;
        }
        G->w[k] = raw_w[k] * (pown / sum);
      }
    }
    for (int64_t k = nreal; k < npoints; ++k) G->w[k] = 0.0;
    *out = G;
    return KLDI_OK;
  });
}

extern "C" kldi_status kldi_grid_info(const kldi_grid* g, int64_t* npoints, int64_t* nreal, int64_t* nblocks) {
  return kldi::guarded("kldi_grid_info", [&]() -> kldi_status {
    if (!g) { kldi::set_error("kldi_grid_info: null grid"); return KLDI_EINVAL; }
    if (npoints) *npoints = g->npoints;
    if (nreal) *nreal = g->nreal;
    if (nblocks) *nblocks = g->nblocks;
    return KLDI_OK;
  });
}

extern "C" kldi_status kldi_grid_export(const kldi_grid* g, double* xyz, double* w, int32_t* atom_of) {
  return kldi::guarded("kldi_grid_export", [&]() -> kldi_status {
    if (!g) { kldi::set_error("kldi_grid_export: null grid"); return KLDI_EINVAL; }
    if (xyz) std::memcpy(xyz, g->xyz.data(), sizeof(double) * g->xyz.size());
    if (w) std::memcpy(w, g->w.data(), sizeof(double) * g->w.size());
    if (atom_of) std::memcpy(atom_of, g->atom.data(), sizeof(int32_t) * g->atom.size());
    return KLDI_OK;
  });
}

namespace {

const char kGridMagic[8] = {'K', 'L', 'D', 'I', 'G', 'R', 'D', '1'};

struct FileCloser {
  FILE* f;
  ~FileCloser() {
    if (f) std::fclose(f);
  }
};

}  // namespace

extern "C" kldi_status kldi_grid_save(const kldi_grid* g, const char* path) {
  return kldi::guarded("kldi_grid_save", [&]() -> kldi_status {
    using namespace kldi;
    if (!g || !path) {
      set_error("kldi_grid_save: null argument");
      return KLDI_EINVAL;
    }
    FILE* f = std::fopen(path, "wb");
    if (!f) {
      set_error("kldi_grid_save: cannot open %s for writing", path);
      return KLDI_EIO;
    }
    const int64_t head[4] = {g->npoints, g->nreal, g->nblocks, (int64_t)g->block};
    bool ok = std::fwrite(kGridMagic, 1, sizeof kGridMagic, f) == sizeof kGridMagic &&
              std::fwrite(head, sizeof(int64_t), 4, f) == 4 &&
              std::fwrite(g->xyz.data(), sizeof(double), g->xyz.size(), f) == g->xyz.size() &&
              std::fwrite(g->w.data(), sizeof(double), g->w.size(), f) == g->w.size() &&
              std::fwrite(g->atom.data(), sizeof(int32_t), g->atom.size(), f) == g->atom.size();
    ok = (std::fclose(f) == 0) && ok;
    if (!ok) {
      std::remove(path);
      set_error("kldi_grid_save: writing %s failed", path);
      return KLDI_EIO;
    }
    return KLDI_OK;
  });
}

extern "C" kldi_status kldi_grid_load(const char* path, kldi_grid** out) {
  return kldi::guarded("kldi_grid_load", [&]() -> kldi_status {
    using namespace kldi;
    if (!path || !out) {
      set_error("kldi_grid_load: null argument");
      return KLDI_EINVAL;
    }
    FileCloser fc{std::fopen(path, "rb")};
    FILE* f = fc.f;
    if (!f) {
      set_error("kldi_grid_load: cannot open %s", path);
      return KLDI_EIO;
    }
    if (std::fseek(f, 0, SEEK_END) != 0) {
      set_error("kldi_grid_load: cannot seek in %s", path);
      return KLDI_EIO;
    }
    const long long flen = (long long)ftello(f);
    std::rewind(f);
    char magic[8];
    int64_t head[4];
    if (flen < 0 || std::fread(magic, 1, sizeof magic, f) != sizeof magic || std::fread(head, sizeof(int64_t), 4, f) != 4) {
      set_error("kldi_grid_load: %s is shorter than the header", path);
      return flen < 0 ? KLDI_EIO : KLDI_EINVAL;
    }
    if (std::memcmp(magic, kGridMagic, sizeof magic) != 0) {
      set_error("kldi_grid_load: %s is not a saved grid", path);
      return KLDI_EINVAL;
    }
    const int64_t npoints = head[0], nreal = head[1], nblocks = head[2], block = head[3];
    if (block != kBlockPts || nblocks <= 0 || nblocks > (INT64_C(1) << 40) / kBlockPts ||
        npoints != nblocks * kBlockPts || nreal <= npoints - kBlockPts || nreal > npoints) {
      set_error("kldi_grid_load: %s: inconsistent sizes (npoints %lld, nreal %lld, nblocks %lld, block %lld)", path,
                (long long)npoints, (long long)nreal, (long long)nblocks, (long long)block);
      return KLDI_EINVAL;
    }
    const long long want = (long long)(sizeof magic + sizeof head) +
                           npoints * (long long)(4 * sizeof(double) + sizeof(int32_t));
    if (flen != want) {
      set_error("kldi_grid_load: %s has %lld bytes, the header implies %lld", path, flen, want);
      return KLDI_EINVAL;
    }
    kldi_grid* G = new kldi_grid;
    std::unique_ptr<kldi_grid> hold(G);
    G->npoints = npoints;
    G->nreal = nreal;
    G->nblocks = nblocks;
    G->xyz.resize(npoints * 3);
    G->w.resize(npoints);
    G->atom.resize(npoints);
    if (std::fread(G->xyz.data(), sizeof(double), G->xyz.size(), f) != G->xyz.size() ||
        std::fread(G->w.data(), sizeof(double), G->w.size(), f) != G->w.size() ||
        std::fread(G->atom.data(), sizeof(int32_t), G->atom.size(), f) != G->atom.size()) {
      set_error("kldi_grid_load: reading %s failed", path);
      return KLDI_EIO;
    }
    for (int64_t k = 0; k < npoints; ++k) {
      const double* p = &G->xyz[k * 3];
      if (!std::isfinite(p[0]) || !std::isfinite(p[1]) || !std::isfinite(p[2]) || !std::isfinite(G->w[k]) ||
          G->atom[k] < 0 || (k >= nreal && G->w[k] != 0.0)) {
        set_error("kldi_grid_load: %s: point %lld is malformed", path, (long long)k);
        return KLDI_EINVAL;
      }
    }
    *out = hold.release();
    return KLDI_OK;
  });
}

extern "C" void kldi_grid_free(kldi_grid* g) { delete g; }

extern "C" const char* kldi_version(void) { return "kldi 0.1 (sm_103a)"; }
