// Basis reordering by overlap signatures (Sec. III-B; appendix "Overlap-Signature
// Construction and Basis-Function Clustering"), host preprocessing run once per
// geometry.  Shells are the units: every function of a Cartesian shell shares
// its centre and exponents, and the kernels evaluate a shell's functions
// together, so a shell's functions stay contiguous.
//
//   signature of shell s:  T_s,t = ||S[s, t]||_F  (Frobenius norm of the overlap block)
//   distance:              d(s, t) = 1 - T_s . T_t / (|T_s| |T_t|)           (cosine, Eq. cosine_distance)
//   clustering:            agglomerative, average linkage: merge the pair of
//                          clusters with the smallest mean leaf distance, then
//                          D(a u b, k) = (n_a D(a, k) + n_b D(b, k)) / (n_a + n_b)
//   orientation:           at each merge the two leaf sequences are reversed or
//                          not so that the closest pair of their end leaves is
//                          adjacent; the root's leaf sequence is the order.
//
// Determinism: sums run sequentially in index order, products are not fused
// (this file is compiled with -ffp-contract=off), the merged pair is the one
// with the smallest (distance, lower id, higher id), the merged cluster keeps
// the lower id and comes first, and the end pairs are tried in the order
// (last, first), (last, last), (first, first), (first, last).
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <vector>

#include "internal.h"

using namespace kldi;

extern "C" kldi_status kldi_order_shells(int nshell, const int* nfn, const double* S, int* perm) {
  return kldi::guarded("kldi_order_shells", [&]() -> kldi_status {
    if (nshell <= 0 || !nfn || !S || !perm) {
      set_error("kldi_order_shells: bad argument");
      return KLDI_EINVAL;
    }
    std::vector<int64_t> off(nshell + 1, 0);
    for (int s = 0; s < nshell; ++s) {
      if (nfn[s] <= 0) {
        set_error("kldi_order_shells: shell %d has %d functions", s, nfn[s]);
        return KLDI_EINVAL;
      }
      off[s + 1] = off[s] + nfn[s];
    }
    const int64_t nbf = off[nshell];
    const int n = nshell;
    // shell signatures
    std::vector<double> T((size_t)n * n);
  #pragma omp parallel for schedule(dynamic, 8)
    for (int s = 0; s < n; ++s)
      for (int t = 0; t < n; ++t) {
        double acc = 0.0;
        for (int64_t mu = off[s]; mu < off[s + 1]; ++mu)
          for (int64_t nu = off[t]; nu < off[t + 1]; ++nu) {
            const double v = S[mu * nbf + nu];
            const double v2 = v * v;
            acc = acc + v2;
          }
        T[(size_t)s * n + t] = std::sqrt(acc);
      }
    std::vector<double> norm(n);
    for (int s = 0; s < n; ++s) {
      double acc = 0.0;
      for (int t = 0; t < n; ++t) {
        const double v = T[(size_t)s * n + t];
        const double v2 = v * v;
        acc = acc + v2;
      }
      norm[s] = std::sqrt(acc);
      if (!(norm[s] > 0.0)) {
        set_error("kldi_order_shells: shell %d has a zero overlap signature", s);
        return KLDI_EINVAL;
      }
    }
    // leaf (shell) cosine distances, and the cluster distance matrix.  The
    // dot products T_s . T_t run over u in order for every t at once (a row of
    // the transposed signatures per u), so each sum has the sequential order.
    std::vector<double> TT((size_t)n * n);
    for (int s = 0; s < n; ++s)
      for (int t = 0; t < n; ++t) TT[(size_t)t * n + s] = T[(size_t)s * n + t];
    std::vector<double> d0((size_t)n * n), D((size_t)n * n);
  #pragma omp parallel
    {
      std::vector<double> acc(n);
  #pragma omp for schedule(dynamic, 4)
      for (int s = 0; s < n; ++s) {
        std::fill(acc.begin(), acc.end(), 0.0);
        for (int u = 0; u < n; ++u) {
          const double a = T[(size_t)s * n + u];
          const double* row = &TT[(size_t)u * n];
          for (int t = 0; t < n; ++t) {
            const double pr = a * row[t];
            acc[t] = acc[t] + pr;
          }
        }
        for (int t = 0; t < n; ++t) {
          const double den = norm[s] * norm[t];
          d0[(size_t)s * n + t] = 1.0 - acc[t] / den;
        }
      }
    }
    D = d0;
    std::vector<char> active(n, 1);
    std::vector<double> size(n, 1.0);
    std::vector<std::vector<int>> leaves(n);
    for (int s = 0; s < n; ++s) leaves[s].push_back(s);
    std::vector<int> nn(n, -1);
    std::vector<double> nd(n, INFINITY);
    auto refresh = [&](int a) {
      nn[a] = -1;
      nd[a] = INFINITY;
      for (int b = 0; b < n; ++b) {
        if (b == a || !active[b]) continue;
        const double v = D[(size_t)a * n + b];
        if (v < nd[a]) {   // equal distances keep the lower id (b increases)
          nd[a] = v;
          nn[a] = b;
        }
      }
    };
    for (int a = 0; a < n; ++a) refresh(a);
    for (int step = 0; step < n - 1; ++step) {
      // the pair with the smallest (distance, lower id, higher id)
      int best = -1;
      for (int a = 0; a < n; ++a) {
        if (!active[a] || nn[a] < 0) continue;
        if (best < 0) { best = a; continue; }
        const int lo_a = std::min(a, nn[a]), hi_a = std::max(a, nn[a]);
        const int lo_b = std::min(best, nn[best]), hi_b = std::max(best, nn[best]);
        if (nd[a] < nd[best] || (nd[a] == nd[best] && (lo_a < lo_b || (lo_a == lo_b && hi_a < hi_b)))) best = a;
      }
      const int p = std::min(best, nn[best]), q = std::max(best, nn[best]);
      // orientation: the closest pair of end leaves becomes adjacent
      std::vector<int>& A = leaves[p];
      std::vector<int>& B = leaves[q];
      const int af = A.front(), al = A.back(), bf = B.front(), bl = B.back();
      const double c[4] = {d0[(size_t)al * n + bf], d0[(size_t)al * n + bl], d0[(size_t)af * n + bf],
                           d0[(size_t)af * n + bl]};
      int k = 0;
      for (int j = 1; j < 4; ++j)
        if (c[j] < c[k]) k = j;
      if (k >= 2) std::reverse(A.begin(), A.end());
      if (k == 1 || k == 3) std::reverse(B.begin(), B.end());
      A.insert(A.end(), B.begin(), B.end());
      B.clear();
      // average linkage
      const double np_ = size[p], nq = size[q];
      active[q] = 0;
      for (int k2 = 0; k2 < n; ++k2) {
        if (!active[k2] || k2 == p) continue;
        const double a1 = np_ * D[(size_t)p * n + k2];
        const double a2 = nq * D[(size_t)q * n + k2];
        const double v = (a1 + a2) / (np_ + nq);
        D[(size_t)p * n + k2] = v;
        D[(size_t)k2 * n + p] = v;
      }
      size[p] = np_ + nq;
      refresh(p);
      for (int k2 = 0; k2 < n; ++k2) {
        if (!active[k2] || k2 == p) continue;
        if (nn[k2] == p || nn[k2] == q) {
          refresh(k2);
        } else {
          const double v = D[(size_t)k2 * n + p];
          if (v < nd[k2] || (v == nd[k2] && p < nn[k2])) {
            nd[k2] = v;
            nn[k2] = p;
          }
        }
      }
    }
    int root = 0;
    while (root < n && !active[root]) ++root;
    for (int s = 0; s < n; ++s) perm[s] = leaves[root][s];
    return KLDI_OK;
  });
}
