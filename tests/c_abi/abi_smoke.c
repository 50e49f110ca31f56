/* The C ABI used from C: one water molecule with a small s/p basis.
 * abi_smoke GRIDFILE [--gpu].  Host-only calls: the grid, its export, the
 * grid saved to GRIDFILE and loaded back, the basis order; with --gpu also
 * kldi_screen and kldi_exc in FP64 and BF16x6, printing E_xc.
 * Built and run by tests/test_c_abi.py. */
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "kldi.h"

static int check(kldi_status st, const char* what) {
  if (st != KLDI_OK) {
    printf("FAIL %s: status %d: %s\n", what, (int)st, kldi_last_error());
    return 1;
  }
  return 0;
}

int main(int argc, char** argv) {
  if (argc < 2) {
    printf("usage: abi_smoke GRIDFILE [--gpu]\n");
    return 2;
  }
  const char* grid_file = argv[1];
  const int gpu = argc > 2 && strcmp(argv[2], "--gpu") == 0;
  const int32_t Z[3] = {8, 1, 1};
  const double xyz[9] = {0.0, 0.0, 0.0, 1.43, 1.11, 0.0, -1.43, 1.11, 0.0};
  const kldi_molecule mol = {3, Z, xyz};
  const int32_t ntheta[1] = {6};
  const kldi_grid_spec spec = {40, 1, ntheta, 128};
  kldi_grid* grid = NULL;
  if (check(kldi_make_grid(&mol, &spec, &grid), "kldi_make_grid")) return 1;
  int64_t np = 0, nreal = 0, nb = 0;
  if (check(kldi_grid_info(grid, &np, &nreal, &nb), "kldi_grid_info")) return 1;
  double* p = malloc(sizeof(double) * 3 * np);
  double* w = malloc(sizeof(double) * np);
  int32_t* at = malloc(sizeof(int32_t) * np);
  if (check(kldi_grid_export(grid, p, w, at), "kldi_grid_export")) return 1;
  /* a normalised-to-pi^(3/2) Gaussian on each atom: the partition of unity
     makes the quadrature of each close to pi^(3/2) */
  double gsum[3] = {0.0, 0.0, 0.0};
  for (int64_t i = 0; i < np; ++i)
    for (int a = 0; a < 3; ++a) {
      const double dx = p[3 * i] - xyz[3 * a], dy = p[3 * i + 1] - xyz[3 * a + 1], dz = p[3 * i + 2] - xyz[3 * a + 2];
      gsum[a] += w[i] * exp(-(dx * dx + dy * dy + dz * dz));
    }
  printf("grid %lld %lld %lld\n", (long long)np, (long long)nreal, (long long)nb);
  printf("gauss %.10f %.10f %.10f\n", gsum[0], gsum[1], gsum[2]);

  /* the grid saved and loaded back: same sizes and the same bytes */
  kldi_grid* loaded = NULL;
  if (check(kldi_grid_save(grid, grid_file), "kldi_grid_save")) return 1;
  if (check(kldi_grid_load(grid_file, &loaded), "kldi_grid_load")) return 1;
  int64_t np2 = 0, nreal2 = 0, nb2 = 0;
  if (check(kldi_grid_info(loaded, &np2, &nreal2, &nb2), "kldi_grid_info (loaded)")) return 1;
  int same = np2 == np && nreal2 == nreal && nb2 == nb;
  if (same) {
    double* p2 = malloc(sizeof(double) * 3 * np);
    double* w2 = malloc(sizeof(double) * np);
    int32_t* at2 = malloc(sizeof(int32_t) * np);
    if (check(kldi_grid_export(loaded, p2, w2, at2), "kldi_grid_export (loaded)")) return 1;
    same = memcmp(p, p2, sizeof(double) * 3 * np) == 0 && memcmp(w, w2, sizeof(double) * np) == 0 &&
           memcmp(at, at2, sizeof(int32_t) * np) == 0;
    free(p2);
    free(w2);
    free(at2);
  }
  kldi_grid_free(loaded);
  kldi_grid* none = NULL;
  const kldi_status missing = kldi_grid_load("", &none);
  printf("reload %s %d\n", same ? "same" : "differs", (int)missing);

  /* basis: O 1s 2s 2p, H 1s on each hydrogen (one primitive each) */
  const int32_t satom[5] = {0, 0, 0, 1, 2}, sl[5] = {0, 0, 1, 0, 0}, snp[5] = {1, 1, 1, 1, 1};
  const double ex[5] = {5.0, 0.5, 0.8, 1.0, 1.0}, co[5] = {1.0, 1.0, 1.0, 1.0, 1.0};
  const kldi_basis basis = {5, satom, sl, snp, ex, co};
  const int nbf = 7;
  /* shell order from an overlap matrix: identity plus a coupling of the two
     hydrogen functions and of the two oxygen s functions */
  double S[49];
  memset(S, 0, sizeof(S));
  for (int i = 0; i < nbf; ++i) S[i * nbf + i] = 1.0;
  S[0 * nbf + 1] = S[1 * nbf + 0] = 0.3;
  S[5 * nbf + 6] = S[6 * nbf + 5] = 0.2;
  const int nfn[5] = {1, 1, 3, 1, 1};
  int perm[5] = {-1, -1, -1, -1, -1};
  if (check(kldi_order_shells(5, nfn, S, perm), "kldi_order_shells")) return 1;
  printf("order %d %d %d %d %d\n", perm[0], perm[1], perm[2], perm[3], perm[4]);
  int bad[5] = {0, -1, 0, 0, 0};
  if (kldi_order_shells(5, bad, S, perm) != KLDI_EINVAL) {
    printf("FAIL kldi_order_shells accepted a shell without functions\n");
    return 1;
  }
  /* the three-atom grid with a one-atom molecule: refused before any device work */
  const kldi_molecule one = {1, Z, xyz};
  const kldi_options opt0 = {1e-12, 1e-12, 1e-14, KLDI_FP64, KLDI_XC_LDA_X, NULL, NULL};
  kldi_plan* none_plan = NULL;
  printf("mismatch %d\n", (int)kldi_screen(grid, &one, &basis, &opt0, &none_plan));

  if (gpu) {
    double D[49];
    memset(D, 0, sizeof(D));
    for (int i = 0; i < nbf; ++i) D[i * nbf + i] = 0.4;
    D[0 * nbf + 1] = D[1 * nbf + 0] = 0.1;
    const int precs[2] = {KLDI_FP64, KLDI_BF16X6};
    for (int k = 0; k < 2; ++k) {
      const kldi_options opt = {1e-12, 1e-12, 1e-14, precs[k], KLDI_XC_LDA_X, NULL, NULL};
      kldi_plan* plan = NULL;
      if (check(kldi_screen(grid, &mol, &basis, &opt, &plan), "kldi_screen")) return 1;
      double V[49], E = 0.0;
      if (check(kldi_exc(plan, KLDI_XC_LDA_X, D, V, &E), "kldi_exc")) return 1;
      double asym = 0.0;
      for (int i = 0; i < nbf; ++i)
        for (int j = 0; j < nbf; ++j) asym = fmax(asym, fabs(V[i * nbf + j] - V[j * nbf + i]));
      printf("exc %d %.15f %.3e %.15f\n", precs[k], E, asym, V[0]);
      kldi_plan_free(plan);
    }
  }
  kldi_grid_free(grid);
  free(p);
  free(w);
  free(at);
  printf("ok\n");
  return 0;
}
