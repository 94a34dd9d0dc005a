// FFT plans: factorisation of M, digit-reversal permutation, twiddle tables.
#include <cmath>
#include <vector>

#include "fft_ct.cuh"
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

struct Shape {
  int id;
  int r[3];
};

// Pass shapes in DIT radix order (see PassShape); longest first.
const Shape kShapes[] = {
    {SH_2_3_3, {2, 3, 3}}, {SH_3_3_3, {3, 3, 3}}, {SH_4_2_3, {4, 2, 3}}, {SH_2_3_5, {2, 3, 5}},
    {SH_4_4_2, {4, 4, 2}}, {SH_2_3, {2, 3, 0}},   {SH_3_3, {3, 3, 0}},   {SH_2_5, {2, 5, 0}},
    {SH_4_3, {4, 3, 0}},   {SH_3_5, {3, 5, 0}},   {SH_4_4, {4, 4, 0}},   {SH_4_5, {4, 5, 0}},
    {SH_5_5, {5, 5, 0}},   {SH_4_2, {4, 2, 0}},   {SH_2, {2, 0, 0}},     {SH_3, {3, 0, 0}},
    {SH_4, {4, 0, 0}},     {SH_5, {5, 0, 0}},
};

}  // namespace

// Group consecutive stages into passes: at each stage take the first (longest)
// shape that matches the next radices with radix product <= maxprod.
void group_passes(FftPlan& p, int k, int maxprod) {
  int t = 0, np = 0;
  while (t < p.nst) {
    int best = -1, blen = 0;
    for (const Shape& sh : kShapes) {
      int len = 0;
      while (len < 3 && sh.r[len] != 0) ++len;
      if (t + len > p.nst) continue;
      int prod = 1;
      for (int q = 0; q < len; ++q) prod *= sh.r[q];
      if (prod > maxprod) continue;
      bool ok = true;
      for (int k = 0; k < len; ++k) ok = ok && (p.R[t + k] == sh.r[k]);
      if (ok && len > blen) {
        best = sh.id;
        blen = len;
      }
    }
    int prod = 1;
    if (best < 0) {
      best = SH_GENERIC;
      blen = 1;
    }
    for (int k = 0; k < blen; ++k) prod *= p.R[t + k];
    p.pshape[k][np] = best;
    p.pR[k][np] = prod;
    p.pLp[k][np] = p.Lp[t];
    p.pdiv[k][np] = make_fastdiv(static_cast<unsigned>(p.Lp[t]));
    ++np;
    t += blen;
  }
  p.npass[k] = np;
  for (int i = np; i < kMaxPasses; ++i) {
    p.pshape[k][i] = SH_2;
    p.pR[k][i] = 1;
    p.pLp[k][i] = 1;
    p.pdiv[k][i] = make_fastdiv(1);
  }
}

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

ghb_status build_plan_tables(int M, FftPlan& p, PlanTables& t) {
  std::vector<int> radices;
  if (M < 1 || !factor(M, radices)) {
    set_error("unsupported transform length M=" + std::to_string(M) +
              " (prime factors must be <= 31)");
    return GHB_ERR_INVALID;
  }
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
  group_passes(p, 0, 18);   // FP64
  group_passes(p, 1, 32);   // FP32

  // perm[n]: write n in mixed radix with the last stage's radix least
  // significant; the position has the digits in stage order, first stage least
  // significant.
  std::vector<int>& perm = t.perm;
  perm.assign(M, 0);
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
  std::vector<double2>& tw64 = t.tw64;
  std::vector<float2>& tw32 = t.tw32;
  tw64.resize(M);
  tw32.resize(M);
  const long double two_pi = 6.283185307179586476925286766559005768L;
  for (int j = 0; j < M; ++j) {
    long double ang = two_pi * static_cast<long double>(j) / static_cast<long double>(M);
    double c = static_cast<double>(cosl(ang));
    double s = -static_cast<double>(sinl(ang));
    tw64[j] = make_double2(c, s);
    tw32[j] = make_float2(static_cast<float>(c), static_cast<float>(s));
  }
  return GHB_OK;
}

ghb_status make_plan(int M, PlanHolder& out) {
  ghb_status st = make_plan_untuned(M, out);
  if (st != GHB_OK) return st;
  return apply_tune(M, out.plan);
}

ghb_status make_plan_untuned(int M, PlanHolder& out) {
  PlanTables t;
  ghb_status st = build_plan_tables(M, out.plan, t);
  if (st != GHB_OK) return st;
  FftPlan& p = out.plan;
  const std::vector<int>& perm = t.perm;
  const std::vector<double2>& tw64 = t.tw64;
  const std::vector<float2>& tw32 = t.tw32;
  GHB_CUDA_TRY(cudaMalloc(&out.d_perm, sizeof(int) * M));
  GHB_CUDA_TRY(cudaMalloc(&out.d_tw64, sizeof(double2) * M));
  GHB_CUDA_TRY(cudaMalloc(&out.d_tw32, sizeof(float2) * M));
  GHB_CUDA_TRY(cudaMemcpy(out.d_perm, perm.data(), sizeof(int) * M, cudaMemcpyHostToDevice));
  GHB_CUDA_TRY(cudaMemcpy(out.d_tw64, tw64.data(), sizeof(double2) * M, cudaMemcpyHostToDevice));
  GHB_CUDA_TRY(cudaMemcpy(out.d_tw32, tw32.data(), sizeof(float2) * M, cudaMemcpyHostToDevice));
  if (ct_size(M) && ct_plan(M).ok) {
    std::vector<int> pct(M);
    ct_perm(M, pct.data());
    GHB_CUDA_TRY(cudaMalloc(&out.d_perm_ct, sizeof(int) * M));
    GHB_CUDA_TRY(cudaMemcpy(out.d_perm_ct, pct.data(), sizeof(int) * M, cudaMemcpyHostToDevice));
  }
  p.perm = out.d_perm;
  p.perm_ct = out.d_perm_ct;
  p.ct_col = p.ct_row = (out.d_perm_ct != nullptr) ? 1 : 0;
  p.tw64 = out.d_tw64;
  p.tw32 = out.d_tw32;
  return GHB_OK;
}

void free_plan(PlanHolder& p) {
  if (p.d_perm) cudaFree(p.d_perm);
  if (p.d_perm_ct) cudaFree(p.d_perm_ct);
  if (p.d_tw64) cudaFree(p.d_tw64);
  if (p.d_tw32) cudaFree(p.d_tw32);
  p = PlanHolder{};
}

}  // namespace ghb
