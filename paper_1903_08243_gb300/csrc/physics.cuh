// Pointwise constitutive kernels shared by the tet and hex vector forms
// (Supplementary material: linear elasticity, St Venant-Kirchhoff; the
// compressible neo-Hookean law is the textbook one).  `gu` is the physical
// displacement gradient of the argument, `gc` that of the linearisation
// point (Jacobian action only); f1[c][j] is the flux that multiplies
// d(phi)/dx_j of test component c.
#pragma once

#include "mfa_internal.h"

namespace mfa {
namespace {

__device__ __forceinline__ double det3(const double A[3][3], double cof[3][3]) {
  cof[0][0] = A[1][1] * A[2][2] - A[1][2] * A[2][1];
  cof[0][1] = A[1][2] * A[2][0] - A[1][0] * A[2][2];
  cof[0][2] = A[1][0] * A[2][1] - A[1][1] * A[2][0];
  cof[1][0] = A[0][2] * A[2][1] - A[0][1] * A[2][2];
  cof[1][1] = A[0][0] * A[2][2] - A[0][2] * A[2][0];
  cof[1][2] = A[0][1] * A[2][0] - A[0][0] * A[2][1];
  cof[2][0] = A[0][1] * A[1][2] - A[0][2] * A[1][1];
  cof[2][1] = A[0][2] * A[1][0] - A[0][0] * A[1][2];
  cof[2][2] = A[0][0] * A[1][1] - A[0][1] * A[1][0];
  return A[0][0] * cof[0][0] + A[0][1] * cof[0][1] + A[0][2] * cof[0][2];
}

// Stress fluxes f1[c][j] multiplying d(phi_a)/dx_j for test component c.
template <int KIND, int LAW>
__device__ __forceinline__ bool physics(const double gu[3][3], const double gc[3][3], double lam, double mu,
                                        double f1[3][3]) {
  if constexpr (KIND == MFA_FORM_ELASTICITY) {
    const double tr = gu[0][0] + gu[1][1] + gu[2][2];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) f1[i][j] = mu * (gu[i][j] + gu[j][i]) + (i == j ? lam * tr : 0.0);
    return true;
  } else if constexpr (KIND == MFA_FORM_HYPER_RES) {
    double F[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) F[i][j] = gu[i][j] + (i == j ? 1.0 : 0.0);
    if constexpr (LAW == MFA_LAW_SVK) {
      // S = lambda tr(E) I + 2 mu E, E = (F^T F - I)/2, P = F S
      double E[3][3];
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = i; j < 3; ++j) {
          const double c = F[0][i] * F[0][j] + F[1][i] * F[1][j] + F[2][i] * F[2][j];
          E[i][j] = 0.5 * (c - (i == j ? 1.0 : 0.0));
          E[j][i] = E[i][j];
        }
      const double tr = E[0][0] + E[1][1] + E[2][2];
      double S[3][3];
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) S[i][j] = 2.0 * mu * E[i][j] + (i == j ? lam * tr : 0.0);
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) f1[i][j] = F[i][0] * S[0][j] + F[i][1] * S[1][j] + F[i][2] * S[2][j];
      return true;
    } else {
      // P = mu F + (lambda ln J - mu) F^{-T},  F^{-T} = cof(F) / J
      double cof[3][3];
      const double J = det3(F, cof);
      if (!(J > 0.0)) return false;
      const double s = (lam * log(J) - mu) / J;
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) f1[i][j] = mu * F[i][j] + s * cof[i][j];
      return true;
    }
  } else {  // MFA_FORM_HYPER_JAC: f1 = dP(F; dF), F = I + gc, dF = gu
    double F[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) F[i][j] = gc[i][j] + (i == j ? 1.0 : 0.0);
    if constexpr (LAW == MFA_LAW_SVK) {
      // dP = dF S + F dS, dE = sym(F^T dF), dS = lambda tr(dE) I + 2 mu dE
      double E[3][3], dE[3][3];
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = i; j < 3; ++j) {
          const double c = F[0][i] * F[0][j] + F[1][i] * F[1][j] + F[2][i] * F[2][j];
          const double d = F[0][i] * gu[0][j] + F[1][i] * gu[1][j] + F[2][i] * gu[2][j] + F[0][j] * gu[0][i] +
                           F[1][j] * gu[1][i] + F[2][j] * gu[2][i];
          E[i][j] = 0.5 * (c - (i == j ? 1.0 : 0.0));
          E[j][i] = E[i][j];
          dE[i][j] = 0.5 * d;
          dE[j][i] = dE[i][j];
        }
      const double tr = E[0][0] + E[1][1] + E[2][2];
      const double dtr = dE[0][0] + dE[1][1] + dE[2][2];
      double S[3][3], dS[3][3];
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
          S[i][j] = 2.0 * mu * E[i][j] + (i == j ? lam * tr : 0.0);
          dS[i][j] = 2.0 * mu * dE[i][j] + (i == j ? lam * dtr : 0.0);
        }
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j)
          f1[i][j] = gu[i][0] * S[0][j] + gu[i][1] * S[1][j] + gu[i][2] * S[2][j] + F[i][0] * dS[0][j] +
                     F[i][1] * dS[1][j] + F[i][2] * dS[2][j];
      return true;
    } else {
      // dP = mu dF + (mu - lambda ln J) A dF^T A + lambda (A : dF) A,  A = F^{-T}
      double cof[3][3];
      const double J = det3(F, cof);
      if (!(J > 0.0)) return false;
      const double iJ = 1.0 / J;
      double A[3][3];
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) A[i][j] = cof[i][j] * iJ;
      double AdFt[3][3];
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) AdFt[i][j] = A[i][0] * gu[j][0] + A[i][1] * gu[j][1] + A[i][2] * gu[j][2];
      double tr = 0.0;
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) tr += A[i][j] * gu[i][j];
      const double c2 = mu - lam * log(J), c3 = lam * tr;
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j)
          f1[i][j] = mu * gu[i][j] + c2 * (AdFt[i][0] * A[0][j] + AdFt[i][1] * A[1][j] + AdFt[i][2] * A[2][j]) +
                     c3 * A[i][j];
      return true;
    }
  }
}

}  // namespace
}  // namespace mfa
