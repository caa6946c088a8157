// Distance scaling of the tight-binding model (Eq. (1), Xu's functional form
// named in Sec. 5): A (r_ref/r)^e exp{e[-(r/r_cut)^ec + (r_ref/r_cut)^ec]}
// for r < r1, a C1 cubic tail on [r1, rm] reaching zero with zero slope at rm,
// and zero beyond.
#pragma once
#include <cmath>
#include "tb.h"

struct tb_gsp {
  double A, rref, e, rcut, ec;   // GSP form
  double r1, rm;                 // tail interval
  double v1, d1, ta, tb;         // tail: v1 + d1 x + ta x^2 + tb x^3, x = r - r1
};

__host__ __device__ inline void tb_gsp_core(const tb_gsp& g, double r, double& v,
                                            double& dv) {
  double pr = pow(r / g.rcut, g.ec);
  v = g.A * pow(g.rref / r, g.e) * exp(g.e * (-pr + pow(g.rref / g.rcut, g.ec)));
  dv = v * (-g.e / r - g.e * g.ec * pr / r);
}

inline tb_gsp tb_make_gsp(double A, double rref, double e, double rcut, double ec,
                          double r1, double rm) {
  tb_gsp g{A, rref, e, rcut, ec, r1, rm, 0, 0, 0, 0};
  tb_gsp_core(g, r1, g.v1, g.d1);
  const double dl = rm - r1;
  g.ta = -(3.0 * g.v1 + 2.0 * g.d1 * dl) / (dl * dl);
  g.tb = (2.0 * g.v1 + g.d1 * dl) / (dl * dl * dl);
  return g;
}

__device__ inline void tb_gsp_eval(const tb_gsp& g, double r, double& v, double& dv) {
  if (r < g.r1) {
    tb_gsp_core(g, r, v, dv);
  } else if (r < g.rm) {
    double x = r - g.r1;
    v = g.v1 + x * (g.d1 + x * (g.ta + x * g.tb));
    dv = g.d1 + x * (2.0 * g.ta + 3.0 * x * g.tb);
  } else {
    v = 0.0;
    dv = 0.0;
  }
}

inline tb_gsp tb_hopping_gsp(const tb_params& p) {
  return tb_make_gsp(1.0, p.r0, p.n, p.rc, p.nc, p.r1, p.rm);
}
inline tb_gsp tb_repulsion_gsp(const tb_params& p) {
  return tb_make_gsp(p.phi0, p.d0, p.m, p.dc, p.mc, p.r1, p.rm);
}
