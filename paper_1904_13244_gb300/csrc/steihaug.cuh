// Steihaug truncated CG (Nocedal & Wright Alg. 7.2; the inner solve of Algorithm 6):
// the float64 scalar and integer slots of the solver's device block and the step
// decision, shared by the launch-per-step form and the persistent column-path form.
#pragma once

#include <cmath>

#include "mrstat.h"

namespace mrstat {

// float64 scalar slots (gn_sc)
enum {
  S_F = 0,       // objective at the trial point / current point
  S_RR,          // res . res
  S_RR_NEW,
  S_GNORM,
  S_MVAL,        // CG model value m(z) - f
  S_COEF,        // step applied to z (alpha_j or tau)
  S_BETA,
  S_DBD, S_RD, S_DD, S_ZD, S_ZZ,  // sums of the step decision (contiguous)
  S_ANORM2,      // ||alpha * mask||^2
  S_GAMMA, S_GAMMA_NEW, S_QQ,     // CGLS
  S_RHOMAX,      // max |rho|
  S_PNORM2,      // z . z after CG
  S_COUNT
};
// integer slots (gn_si)
enum { I_ACTIVE = 0, I_CONT, I_EXIT, I_STEPS, I_FROZEN, I_MASKCOUNT, I_COUNT };

__device__ __forceinline__ double to_boundary(double zz, double zd, double dd, double delta) {
  const double disc = fmax(zd * zd + dd * (delta * delta - zz), 0.0);
  return (-zd + sqrt(disc)) / dd;
}

// One Steihaug decision (Nocedal & Wright Alg. 7.2): choose the step along dir.
__device__ __forceinline__ void st_step(double* sc, int* si, double delta) {
  const double dBd = sc[S_DBD], rd = sc[S_RD], dd = sc[S_DD], zd = sc[S_ZD], zz = sc[S_ZZ];
  si[I_STEPS] += 1;
  if (!(dBd > 0.0)) {
    const double tau = to_boundary(zz, zd, dd, delta);
    sc[S_MVAL] += tau * rd + 0.5 * tau * tau * dBd;
    sc[S_COEF] = tau;
    si[I_CONT] = 0;
    si[I_ACTIVE] = 0;
    si[I_EXIT] = MRSTAT_CG_NEGATIVE_CURVATURE;
    return;
  }
  const double a = sc[S_RR] / dBd;
  const double zn2 = zz + 2.0 * a * zd + a * a * dd;
  if (sqrt(fmax(zn2, 0.0)) >= delta) {
    const double tau = to_boundary(zz, zd, dd, delta);
    sc[S_MVAL] += tau * rd + 0.5 * tau * tau * dBd;
    sc[S_COEF] = tau;
    si[I_CONT] = 0;
    si[I_ACTIVE] = 0;
    si[I_EXIT] = MRSTAT_CG_BOUNDARY;
    return;
  }
  sc[S_MVAL] += a * rd + 0.5 * a * a * dBd;
  sc[S_COEF] = a;
  si[I_CONT] = 1;
}

// tolerance and iteration-count test after a continuing step; beta for the next direction
__device__ __forceinline__ void st_beta(double* sc, int* si, double rel_tol, int max_steps) {
  const double rr_new = sc[S_RR_NEW];
  if (sqrt(rr_new) <= rel_tol * sc[S_GNORM]) {
    si[I_ACTIVE] = 0;
    si[I_CONT] = 0;
    si[I_EXIT] = MRSTAT_CG_CONVERGED;
    return;
  }
  sc[S_BETA] = rr_new / sc[S_RR];
  sc[S_RR] = rr_new;
  if (si[I_STEPS] >= max_steps) {
    si[I_ACTIVE] = 0;
    si[I_CONT] = 0;
    si[I_EXIT] = MRSTAT_CG_MAX_ITER;
  }
}

}  // namespace mrstat
