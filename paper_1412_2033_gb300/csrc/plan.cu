// FFT plans: factorisation of M, digit-reversal permutation, twiddle tables.
#include <cmath>
#include <vector>

#include "ghb_internal.cuh"

namespace ghb {

namespace {

bool factor(int M, std::vector<int>& radices) {
  radices.clear();
  int m = M;
  while (m % 4 == 0) { radices.push_back(4); m /= 4; }
  while (m % 2 == 0) { radices.push_back(2); m /= 2; }
  while (m % 3 == 0) { radices.push_back(3); m /= 3; }
  while (m % 5 == 0) { radices.push_back(5); m /= 5; }
  for (int p = 7; p <= kMaxGenericRadix && m > 1; p += 2) {
    while (m % p == 0) { radices.push_back(p); m /= p; }
  }
  return m == 1 && static_cast<int>(radices.size()) <= kMaxStages;
}

}  // namespace

bool factorizable(int M) {
  std::vector<int> r;
  return M >= 1 && factor(M, r);
}

// Smallest M >= 2N - 1 with prime factors 2, 3, 5 only (Lemma integ_eval_VM
// allows any M >= 2N - 1; 5-smooth sizes keep every stage a specialised radix).
int auto_M(int N) {
  for (int M = 2 * N - 1;; ++M) {
    int m = M;
    for (int p : {2, 3, 5}) while (m % p == 0) m /= p;
    if (m == 1) return M;
  }
}

ghb_status make_plan(int M, PlanHolder& out) {
  std::vector<int> radices;
  if (M < 1 || !factor(M, radices)) {
    set_error("unsupported transform length M=" + std::to_string(M) +
              " (prime factors must be <= 31)");
    return GHB_ERR_INVALID;
  }
  FftPlan& p = out.plan;
  p = FftPlan{};
  p.M = M;
  p.nst = static_cast<int>(radices.size());
  int L = 1;
  for (int t = 0; t < p.nst; ++t) {
    p.R[t] = radices[t];
    p.Lp[t] = L;
    L *= radices[t];
  }
  for (int t = p.nst; t < kMaxStages; ++t) { p.R[t] = 1; p.Lp[t] = L; }

  // perm[n]: write n in mixed radix with the last stage's radix least
  // significant; the position has the digits in stage order, first stage least
  // significant.
  std::vector<int> perm(M);
  std::vector<int> q(p.nst > 0 ? p.nst : 1);
  for (int n = 0; n < M; ++n) {
    int rem = n;
    for (int t = p.nst - 1; t >= 0; --t) {
      q[t] = rem % p.R[t];
      rem /= p.R[t];
    }
    int pos = 0;
    for (int t = 0; t < p.nst; ++t) pos += q[t] * p.Lp[t];
    perm[n] = pos;
  }
  std::vector<double2> tw64(M);
  std::vector<float2> tw32(M);
  const long double two_pi = 6.283185307179586476925286766559005768L;
  for (int j = 0; j < M; ++j) {
    long double ang = two_pi * static_cast<long double>(j) / static_cast<long double>(M);
    double c = static_cast<double>(cosl(ang));
    double s = -static_cast<double>(sinl(ang));
    tw64[j] = make_double2(c, s);
    tw32[j] = make_float2(static_cast<float>(c), static_cast<float>(s));
  }
  GHB_CUDA_TRY(cudaMalloc(&out.d_perm, sizeof(int) * M));
  GHB_CUDA_TRY(cudaMalloc(&out.d_tw64, sizeof(double2) * M));
  GHB_CUDA_TRY(cudaMalloc(&out.d_tw32, sizeof(float2) * M));
  GHB_CUDA_TRY(cudaMemcpy(out.d_perm, perm.data(), sizeof(int) * M, cudaMemcpyHostToDevice));
  GHB_CUDA_TRY(cudaMemcpy(out.d_tw64, tw64.data(), sizeof(double2) * M, cudaMemcpyHostToDevice));
  GHB_CUDA_TRY(cudaMemcpy(out.d_tw32, tw32.data(), sizeof(float2) * M, cudaMemcpyHostToDevice));
  p.perm = out.d_perm;
  p.tw64 = out.d_tw64;
  p.tw32 = out.d_tw32;
  return GHB_OK;
}

void free_plan(PlanHolder& p) {
  if (p.d_perm) cudaFree(p.d_perm);
  if (p.d_tw64) cudaFree(p.d_tw64);
  if (p.d_tw32) cudaFree(p.d_tw32);
  p = PlanHolder{};
}

}  // namespace ghb
