/*
 * Brute-force partition function of a small periodic lattice.
 *
 * TEST INFRASTRUCTURE ONLY: part of the oracle; never linked into the CUDA
 * library.
 *
 * Z = sum over all q^(Lx*Ly) spin configurations of
 *     prod_sites w[s_i] * prod_{2 Lx Ly bonds} B[s_i, s_j]
 * on an Lx x Ly torus where every site owns the bond to its right neighbour
 * and the bond to its upper neighbour (periodic), i.e. Z = Tr T^N of Eq. (2)
 * written in the spin variables.  Terms are summed in log space against the
 * largest term, in long double.
 */
#include <math.h>
#include <stdlib.h>

static long double config_log_weight(int q, int Lx, int Ly, const int *s,
                                     const double *lnB, const double *lnw) {
  long double e = 0.0L;
  for (int i = 0; i < Lx; ++i) {
    for (int j = 0; j < Ly; ++j) {
      int a = s[i * Ly + j];
      int right = s[((i + 1) % Lx) * Ly + j];
      int up = s[i * Ly + (j + 1) % Ly];
      e += lnw[a] + lnB[a * q + right] + lnB[a * q + up];
    }
  }
  return e;
}

/* Returns ln Z, or NAN on invalid input (non-positive weights, too many states). */
double oracle_brute_ln_z(int q, int Lx, int Ly, const double *B, const double *w) {
  int N = Lx * Ly;
  if (q < 1 || q > 8 || Lx < 1 || Ly < 1 || N > 24) return NAN;
  long long total = 1;
  for (int i = 0; i < N; ++i) {
    total *= q;
    if (total > 400000000LL) return NAN;
  }
  double lnB[64], lnw[8];
  for (int a = 0; a < q; ++a) {
    if (!(w[a] > 0.0)) return NAN;
    lnw[a] = log(w[a]);
    for (int b = 0; b < q; ++b) {
      if (!(B[a * q + b] > 0.0)) return NAN;
      lnB[a * q + b] = log(B[a * q + b]);
    }
  }
  int *s = (int *)calloc((size_t)N, sizeof(int));
  if (!s) return NAN;
  long double emax = -INFINITY;
  for (int pass = 0; pass < 2; ++pass) {
    long double acc = 0.0L;
    for (int i = 0; i < N; ++i) s[i] = 0;
    for (long long c = 0; c < total; ++c) {
      long double e = config_log_weight(q, Lx, Ly, s, lnB, lnw);
      if (pass == 0) {
        if (e > emax) emax = e;
      } else {
        acc += expl(e - emax);
      }
      for (int i = 0; i < N; ++i) { /* odometer increment */
        if (++s[i] < q) break;
        s[i] = 0;
      }
    }
    if (pass == 1) {
      free(s);
      return (double)(emax + logl(acc));
    }
  }
  free(s);
  return NAN;
}
