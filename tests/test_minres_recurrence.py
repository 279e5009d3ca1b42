"""The per-RHS scalar recurrence of the coarse MINRES (csrc/minres.cuh: the
Givens QR of the Lanczos tridiagonal and the update coefficients), built for
the host and driven by a harness that takes the Lanczos and update vector
steps exactly as the coarse kernels do (z = A v - alpha v - beta v_prev,
w = cf0 v + cf1 w1 + cf2 w2, x += cf3 w, v_next = cf4 z) on a small complex
Hermitian indefinite matrix.  Pinned against the mathematics of MINRES: the
recurrence's |eta| equals the true residual |b - A x_k| at every iteration,
that residual never grows, and after n iterations x equals numpy's solution."""
import os
import shutil
import subprocess

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "..", "paper_2412_06347_gb300", "csrc")
CUDA_INC = "/usr/local/cuda/include"

PROG = r"""
#include <complex>
#include <cstdio>
#include <vector>
#include "minres.cuh"
using namespace mglma;
typedef std::complex<double> C;
int main() {
  int n, iters;
  if (std::scanf("%d %d", &n, &iters) != 2) return 1;
  std::vector<C> A(n * n), b(n);
  for (auto& a : A) { double re, im; std::scanf("%lf %lf", &re, &im); a = C(re, im); }
  for (auto& v : b) { double re, im; std::scanf("%lf %lf", &re, &im); v = C(re, im); }
  const int cap = 1;
  std::vector<double> st(MR_COUNT * cap, 0.0);
  auto S = [&](int j) -> double& { return st[j]; };
  int active = 1;
  // initialisation as the library's (v_0 = b / beta_1, zero directions)
  double bb = 0;
  for (auto& v : b) bb += std::norm(v);
  S(MR_BB) = bb;
  const double b1 = std::sqrt(bb);
  S(MR_BETA1) = b1; S(MR_ETA) = b1; S(MR_BETA) = 0; S(MR_C2) = S(MR_C1) = 1; S(MR_S2) = S(MR_S1) = 0;
  std::vector<C> v(n), vo(n, 0.0), z(n), w1(n, 0.0), w2(n, 0.0), x(n, 0.0);
  for (int i = 0; i < n; ++i) v[i] = b[i] / b1;
  for (int k = 0; k < iters && active; ++k) {
    for (int i = 0; i < n; ++i) { z[i] = 0; for (int j = 0; j < n; ++j) z[i] += A[i * n + j] * v[j]; }
    C dotc = 0;
    for (int i = 0; i < n; ++i) dotc += std::conj(v[i]) * z[i];
    const double2 dot = make_double2(dotc.real(), dotc.imag());
    double zz = 0;
    for (int i = 0; i < n; ++i) { z[i] = z[i] - dotc.real() * v[i] - S(MR_BETA) * vo[i]; zz += std::norm(z[i]); }
    S(MR_BN2) = zz;
    minres_scalar_step(st.data(), &dot, &active, 0.0, cap, 0);
    if (S(MR_CF + 5) != 0.0) {
      std::vector<C> wn(n);
      for (int i = 0; i < n; ++i) {
        wn[i] = S(MR_CF) * v[i] + S(MR_CF + 1) * w1[i] + S(MR_CF + 2) * w2[i];
        x[i] += S(MR_CF + 3) * wn[i];
      }
      w2 = w1; w1 = wn;
      vo = v;
      for (int i = 0; i < n; ++i) v[i] = S(MR_CF + 4) * z[i];
    }
    std::printf("eta %d %.17g\n", k, std::fabs(S(MR_ETA)));
    for (int i = 0; i < n; ++i) std::printf("x %d %d %.17g %.17g\n", k, i, x[i].real(), x[i].imag());
  }
  return 0;
}
"""


@pytest.fixture(scope="module")
def exe(tmp_path_factory):
    gxx = shutil.which("g++")
    if not gxx or not os.path.isfile(os.path.join(CUDA_INC, "cuda_runtime.h")):
        pytest.skip("g++ or the CUDA headers are missing")
    d = tmp_path_factory.mktemp("minres")
    src, out = d / "minres_test.cpp", d / "minres_test"
    src.write_text(PROG)
    subprocess.run([gxx, "-std=c++17", "-O2", "-I", CSRC, "-I", CUDA_INC, str(src), "-o", str(out)], check=True,
                   capture_output=True)
    return str(out)


def _run(exe, A, b, iters):
    n = len(b)
    vals = [f"{n} {iters}"] + [f"{a.real:.17g} {a.imag:.17g}" for a in A.ravel()] + \
        [f"{v.real:.17g} {v.imag:.17g}" for v in b]
    out = subprocess.run([exe], input="\n".join(vals), check=True, capture_output=True, text=True).stdout
    eta, xs = {}, {}
    for ln in out.splitlines():
        t = ln.split()
        if t[0] == "eta":
            eta[int(t[1])] = float(t[2])
        else:
            xs.setdefault(int(t[1]), np.zeros(n, complex))[int(t[2])] = float(t[3]) + 1j * float(t[4])
    return eta, xs


def _hermitian_indefinite(n, seed):
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.normal(size=(n, n)) + 1j * rng.normal(size=(n, n)))
    lam = np.concatenate([rng.uniform(0.3, 2.0, n - n // 3), -rng.uniform(0.3, 2.0, n // 3)])
    A = (Q * lam) @ Q.conj().T
    return (A + A.conj().T) / 2, rng.normal(size=n) + 1j * rng.normal(size=n)


def test_eta_is_the_true_residual_and_never_grows(exe):
    A, b = _hermitian_indefinite(24, 5)
    eta, xs = _run(exe, A, b, 24)
    nb = np.linalg.norm(b)
    prev = np.inf
    for k in sorted(eta):
        res = np.linalg.norm(b - A @ xs[k])
        assert abs(eta[k] - res) <= 1e-10 * nb, (k, eta[k], res)
        assert res <= prev * (1 + 1e-12) + 1e-13 * nb
        prev = res


def test_solution_after_n_iterations(exe):
    A, b = _hermitian_indefinite(16, 9)
    eta, xs = _run(exe, A, b, 16)
    x = xs[max(xs)]
    assert np.linalg.norm(x - np.linalg.solve(A, b)) <= 1e-9 * np.linalg.norm(np.linalg.solve(A, b))
