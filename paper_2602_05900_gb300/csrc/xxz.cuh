// Two-site operators of the spin-1/2 XXZ chain h = Jxy (Sx Sx + Sy Sy) + Jz Sz Sz
// (Jxy = Jz = J: the Heisenberg chain of Sec. II.A) in closed form, host side.
// Basis of a site: 0 = Sz +1/2, 1 = Sz -1/2; a two-site state (a, b) has index
// 2 a + b; matrices are row-major 4 x 4, [out][in].
#pragma once

#include <math.h>

namespace hotrg {

// h: diagonal Jz/4 on |00>, |11> and -Jz/4 on |01>, |10>; Jxy/2 between |01> and |10>
inline void xxz_bond_h(double Jxy, double Jz, double h[16]) {
  for (int i = 0; i < 16; ++i) h[i] = 0.0;
  h[0] = h[15] = 0.25 * Jz;
  h[5] = h[10] = -0.25 * Jz;
  h[6] = h[9] = 0.5 * Jxy;
}

// g = exp(-tau h) from the spectrum of h: |00>, |11> -> Jz/4,
// (|01> + |10>)/sqrt2 -> Jxy/2 - Jz/4, (|01> - |10>)/sqrt2 -> -Jxy/2 - Jz/4
inline void xxz_gate(double Jxy, double Jz, double tau, double g[16]) {
  const double p = exp(-0.25 * tau * Jz);
  const double es = exp(-tau * (0.5 * Jxy - 0.25 * Jz)), ea = exp(-tau * (-0.5 * Jxy - 0.25 * Jz));
  for (int i = 0; i < 16; ++i) g[i] = 0.0;
  g[0] = g[15] = p;
  g[5] = g[10] = 0.5 * (es + ea);
  g[6] = g[9] = 0.5 * (es - ea);
}

}  // namespace hotrg
