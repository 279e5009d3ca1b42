// Per-RHS scalar recurrence of the batched coarse MINRES (Givens QR of the
// Lanczos tridiagonal), shared by its own kernel and by the Lanczos-norm
// kernel that runs it in its last block.  State layout: st[j * cap + r] for
// the slots below.
#pragma once
#include <cuda_runtime.h>

#include <cmath>

namespace mglma {

enum {
  MR_BETA1 = 0,
  MR_ETA,
  MR_BETA,
  MR_C2,
  MR_S2,
  MR_C1,
  MR_S1,
  MR_BN2,
  MR_BB,
  MR_CF,  // six update coefficients (minres_update), MR_CF + 4 also scales v_0
  MR_COUNT = MR_CF + 6
};

// alpha = Re dot[r] = <v_k, Qhat v_k>, |z|^2 in slot MR_BN2: the rotation of
// iteration k, the update coefficients (MR_CF .. MR_CF + 5; MR_CF + 5 = 1
// when the update applies) and the new activity of RHS r
__host__ __device__ __forceinline__ void minres_scalar_step(double* st, const double2* dot, int* active, double tol,
                                                            int cap, int r) {
  auto S = [&](int j) -> double& { return st[(size_t)j * cap + r]; };
  S(MR_CF + 5) = 0;
  if (!active[r]) return;
  const double alpha = dot[r].x, beta = S(MR_BETA);
  const double bn = sqrt(fmax(S(MR_BN2), 0.0));
  const double eps = S(MR_S2) * beta, dp = S(MR_C2) * beta;
  const double delta = S(MR_C1) * dp + S(MR_S1) * alpha;
  const double gp = S(MR_C1) * alpha - S(MR_S1) * dp;
  const double gamma = hypot(gp, bn);
  if (!(gamma > 0) || !(gamma < INFINITY)) {  // breakdown: keep the iterate
    active[r] = 0;
    return;
  }
  const double c = gp / gamma, sn = bn / gamma;
  S(MR_CF + 0) = 1.0 / gamma;
  S(MR_CF + 1) = -delta / gamma;
  S(MR_CF + 2) = -eps / gamma;
  S(MR_CF + 3) = c * S(MR_ETA);
  S(MR_CF + 4) = bn > 0 ? 1.0 / bn : 0.0;
  S(MR_CF + 5) = 1;
  S(MR_ETA) = -sn * S(MR_ETA);
  S(MR_C2) = S(MR_C1);
  S(MR_S2) = S(MR_S1);
  S(MR_C1) = c;
  S(MR_S1) = sn;
  S(MR_BETA) = bn;
  active[r] = (bn > 0 && fabs(S(MR_ETA)) > tol * S(MR_BETA1)) ? 1 : 0;
}

}  // namespace mglma
