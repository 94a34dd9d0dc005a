// Internal declarations of the ghb library (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <string>
#include <vector>

#include "fft.cuh"
#include "ghb.h"

namespace ghb {

// ---------------------------------------------------------------------------
// error plumbing
// ---------------------------------------------------------------------------
void set_error(const std::string& msg);

#define GHB_CUDA_TRY(expr)                                                     \
  do {                                                                         \
    cudaError_t err__ = (expr);                                                \
    if (err__ != cudaSuccess) {                                                \
      ::ghb::set_error(std::string(#expr) + ": " + cudaGetErrorString(err__)); \
      return err__ == cudaErrorMemoryAllocation ? GHB_ERR_OOM : GHB_ERR_CUDA;  \
    }                                                                          \
  } while (0)

// Return a failing ghb_status from the enclosing function.
#define TRY_STATUS(expr)                 \
  do {                                   \
    const ghb_status st__ = (expr);      \
    if (st__ != GHB_OK) return st__;     \
  } while (0)

// ---------------------------------------------------------------------------
// device-side CG scalars (one per running solve)
// ---------------------------------------------------------------------------
enum DoneCode { RUNNING = 0, CONVERGED = 1, BREAKDOWN = 2, MAXITER = 3 };

struct CgState {
  double rr;       // <r, r> (full-spectrum inner product)
  double pq;       // <p, A p>
  double alpha;
  double beta;
  double bb;       // <b, b>
  double tol2;     // stop when rr <= tol2 (= tol^2 bb)
  int iter;
  int maxiter;
  int done;        // DoneCode
  int pad;
  unsigned int ticket;  // last-block counter of the running reduction
  unsigned int pad2;
  // bound tracking (Section 7.4): dec = sum_{j<iter} alpha_j <r_j, r_j>, the
  // decrease of the energy along the CG iterates, J(x_i) = J(x_0) - dec_i;
  // written to hist[i] for i < hist_cap when hist is not null
  double dec;
  double* hist;
  int hist_cap;
  int pad3;
};

constexpr int kMaxPartials = 4096;

// Relative reduction asked of an FP32 inner solve that starts from the FP64
// residual <r, r> = rr of a solve with <b, b> = bb and outer tolerance tol:
// inner_tol, or half of what the outer tolerance still needs when that is
// less (so a last correction that only has to gain a small factor takes a
// few FP32 iterations instead of a full inner_tol reduction), at most 1/2.
inline double inner_target(double inner_tol, double tol, double rr, double bb) {
  if (!(rr > 0.0) || !(bb > 0.0)) return inner_tol;
  const double need = 0.5 * tol * std::sqrt(bb / rr);
  return std::min(0.5, std::max(inner_tol, need));
}

// ---------------------------------------------------------------------------
// inclusions on the device
// ---------------------------------------------------------------------------
struct Incl {
  int shape;
  int pad;
  double c[3];
  double s[3];
  double dv;       // (inside value - matrix value) of the coefficient tabulated
  double v;        // the inside value itself (point samples of the GaNi scheme)
};

// ---------------------------------------------------------------------------
// geometry of one context
// ---------------------------------------------------------------------------
struct Geometry {
  int d;
  int N[3];
  int M[3];
  int h;                  // (N_d + 1)/2: stored half of the last axis
  int64_t P;              // complex entries per component of a field
  int64_t field;          // d * P
  int64_t T1;             // entries of the axis-1 intermediate (all components)
  int64_t T2;             // entries of the axis-2 intermediate (d = 3)
  int64_t rows;           // rows of the last-axis pass: M_1 (d=2), M_1 M_2 (d=3)
  int64_t grid;           // |M|
  int64_t table;          // entries of the half table on Z_{2N-1}
};

// Host-owned plan with its device tables.
struct PlanHolder {
  FftPlan plan{};
  int* d_perm = nullptr;
  int* d_perm_ct = nullptr;
  double2* d_tw64 = nullptr;
  float2* d_tw32 = nullptr;
};

// Plan with tables on the device and the autotuned launch configuration
// (make_plan) or the size rules (make_plan_untuned).
ghb_status make_plan(int M, PlanHolder& out);
ghb_status make_plan_untuned(int M, PlanHolder& out);
// Regroup the stages of precision k ([0] FP64, [1] FP32) into passes of radix
// product <= maxprod.
void group_passes(FftPlan& p, int k, int maxprod);
// Write the autotuned configuration for length M into p (tuning M first if
// it has not been tuned in this process and tuning is enabled).
ghb_status apply_tune(int M, FftPlan& p);
// Host tables of a plan (digit reversal, twiddles); the
// plan's device pointers are left null for the caller to place the tables.
struct PlanTables {
  std::vector<int> perm;
  std::vector<double2> tw64;
  std::vector<float2> tw32;
};
ghb_status build_plan_tables(int M, FftPlan& p, PlanTables& t);
void free_plan(PlanHolder& p);
bool factorizable(int M);
int auto_M(int N);

// ---------------------------------------------------------------------------
// launchers (kernels.cu)
// ---------------------------------------------------------------------------
enum ColMode { COL_PLAIN = 0, COL_PUPDATE = 1 };

// Column pass: transforms along a non-contiguous axis.  Arrays are viewed as
// [outer][L][inner]; `in` has L = Lin, `out` has L = Lout.
//  sign = +1: zero-pad (input index i is frequency i - (Lin-1)/2), inverse DFT
//             of length M, output rows m = 0..M-1 (Lout = M).
//  sign = -1: forward DFT of the M input rows, keep frequencies of Z_Lout
//             (centred), scale by 1/M.
struct ColArgs {
  const void* in;
  void* out;
  const void* pold;   // COL_PUPDATE: p_old (read), written back as p = in + beta p_old
  void* pnew;
  const CgState* st;  // COL_PUPDATE: beta; early exit when done
  int64_t outer, inner;
  int Lin, Lout;
};

template <typename T>
ghb_status launch_col(int sign, int mode, const ColArgs& a, const FftPlan& pl, cudaStream_t s);

enum RowMode { ROW_MATVEC = 0, ROW_TOREAL = 1, ROW_ENERGY = 2 };

// Row pass along the contiguous half-spectrum axis.
struct RowArgs {
  void* t[3];          // per field: [c][row][H] complex half spectra (MATVEC: in place)
  int nfields;
  int ncomp;           // components per field
  int64_t rows;
  int H;               // stored half length (h for fields, N_d for the table)
  int64_t comp_stride; // entries between components (= rows * H)
  const void* a;       // [row][M] real multiplier (MATVEC, ENERGY)
  void* out_real;      // [row][M] real output (TOREAL)
  double* partials;    // ENERGY: per-block partial Gram
  double* gram;        // ENERGY: final Gram (nfields^2), scaled by 1/|M|
  unsigned int* ticket;
  double scale;        // ENERGY: 1/|M|
  const CgState* st;   // MATVEC: early exit when done (may be null)
};

template <typename T>
ghb_status launch_row(int mode, const RowArgs& a, const FftPlan& pl, cudaStream_t s);

// Work items of batched launches: every item is one operand (an instance's
// solve) with its own sizes and plan; it owns blocks [block_begin, block_begin + nblocks).
struct ColItem {
  ColArgs a;
  const FftPlan* pl;     // device copy of the item's plan
  int64_t block_begin;
};

struct RowItem {
  RowArgs a;
  const FftPlan* pl;
  int rows_per_cta;
  int pad;
  int64_t nblocks;
  int64_t block_begin;
};

// Batched launches; TW / NL and the shared-memory size are chosen by the caller
// for the largest M of the batch (col_tile_width, row_lines).
template <typename T>
ghb_status launch_col_batch(int sign, int mode, int TW, const ColItem* items, int n, int64_t blocks,
                            size_t smem, int threads, cudaStream_t s);
template <typename T>
ghb_status launch_row_batch(int mode, int NL, const RowItem* items, int n, int64_t blocks, size_t smem, int threads,
                            cudaStream_t s);
// rows per CTA and interleaved complex lines of a row pass
// Rows per CTA and interleaved complex lines of a last-axis pass; rows32 is the
// plan's tuned row count of the FP32 2-D operator (0 = size rule).
void row_lines(int mode, int nfields, int ncomp, int M, int rows32, int* rows_per_cta, int* NL);

// Field-level kernels (half-spectrum fields of one context).
struct FieldGeom {
  int d;
  int N[3];
  int h;
  int64_t P;
  FastDiv hdiv;    // division by h (entry index -> row, j)
  FastDiv n1div;   // division by N[1] (row -> i_1, i_2 for d = 3)
};

// Field geometry with its divisors: the field kernels split an entry index
// into (row, j) and a row into (i_1, i_2) by multiply-high division, since a
// run-time integer division costs tens of instructions per entry.
inline FieldGeom make_field_geom(int d, int N0, int N1, int N2, int h, int64_t P) {
  FieldGeom f;
  f.d = d;
  f.N[0] = N0;
  f.N[1] = N1;
  f.N[2] = N2;
  f.h = h;
  f.P = P;
  f.hdiv = make_fastdiv(static_cast<unsigned>(h > 0 ? h : 1));
  f.n1div = make_fastdiv(static_cast<unsigned>(N1 > 0 ? N1 : 1));
  return f;
}

// Coefficient tables on Z_{2N-1} (eq. inclcomp_formula) of the inclusion lists
// incs0 and, when tab1 is not null, incs1 (same shapes and centres, other jumps:
// the coefficient 1/a beside a), each list's background value a0v0 / a0v1.
ghb_status launch_coeff_tables(double2* tab0, double2* tab1, const Geometry& g, const Incl* incs0,
                               const Incl* incs1, int n, double a0v0, double a0v1, cudaStream_t s);
template <typename T>
ghb_status launch_rhs(void* b, const double2* tab, const Geometry& g, const double* E, int kind,
                      cudaStream_t s);
template <typename T>
ghb_status launch_project(void* y, const void* w, const FieldGeom& fg, int kind, cudaStream_t s);
template <typename T>
ghb_status launch_cg_init(void* x, void* r, void* p, const void* b, const FieldGeom& fg, CgState* st,
                          double* partials, double tol, int maxiter, cudaStream_t s);
template <typename T>
ghb_status launch_project_dot(void* q, const void* w, const void* p, const FieldGeom& fg, int kind,
                              CgState* st, double* partials, cudaStream_t s);
template <typename T>
ghb_status launch_update(void* x, void* r, const void* p, const void* q, const FieldGeom& fg,
                         CgState* st, double* partials, cudaStream_t s);
// r64 = b64 - y64, rr into st (FP64 outer residual); also st->done reset
// Fields of a Gram matrix on Z_N: v[i] = E_i + x_i (admissible fields, with
// the load at k = 0) and y[i] the operator output of x_i before projection.
struct GramZnArgs {
  const double2* v[3];
  const double2* y[3];
};
// X_ij = Re sum_{k in Z_N} (a^ E_i + y_i)(k) . conj v_j(k) (d x d, row-major)
// into out (device, d^2 doubles); partials holds max_partials doubles.
ghb_status launch_gram_zn(const GramZnArgs& ga, const double2* tab, const Geometry& g, double* partials,
                          int max_partials, double* out, cudaStream_t s);
ghb_status launch_residual(double2* r, const double2* b, const double2* y, const FieldGeom& fg,
                           CgState* st, double* partials, cudaStream_t s);
ghb_status launch_to_f32(float2* dst, const double2* src, const FieldGeom& fg, cudaStream_t s);
// x = base + (double) dx
ghb_status launch_accum_f32(double2* x, const double2* base, const float2* dx, const FieldGeom& fg,
                            cudaStream_t s);

// CG vector operations over many operands in one launch.
enum CgOp { CG_INIT = 0, CG_PROJECT_DOT, CG_UPDATE, CG_PROJECT, CG_RESIDUAL, CG_TO_F32, CG_ACCUM };
struct CgItem {
  FieldGeom fg;
  void* x;
  void* r;
  void* p;
  void* q;
  const void* w;
  const void* b;
  CgState* st;
  double* partials;   // at least nblocks doubles
  int kind;
  int maxiter;
  double tol;
  int64_t nblocks;
  int64_t block_begin;
};
// blocks a one-operand launch of the CG vector operations uses for this field
int64_t cg_blocks(const FieldGeom& fg);
template <typename T>
ghb_status launch_cg_batch(int op, const CgItem* items, int n, int64_t blocks, cudaStream_t s);
ghb_status launch_to_f32_real(float* dst, const double* src, int64_t n, cudaStream_t s);
// Point samples a(x^k), x^k = k / N (k_a = 0..N_a-1, C-order), of a0 + inclusions
// (the GaNi scheme's data, eq. approx_bilin): FP64 and an FP32 copy.
ghb_status launch_sample_values(double* out64, float* out32, const Geometry& g, const Incl* incs, int n,
                                double a0v, cudaStream_t s);
// Table of a pixel image (Lemma grid_compos with the pixel characteristic
// function): tab(m) = prod_a sinc(m_a / P_a) Chat((m_a + (P_a - 1)/2) mod P_a),
// m in Z_{2N-1} (half table); Chat = the image's normalised DFT with frequency
// i - (P_a - 1)/2 at index i (the forward column pass with Lout = P_a).
ghb_status launch_image_table(double2* tab, const Geometry& g, const double2* chat, const int* P, cudaStream_t s);
// Reduced Ga operator (Lemma reduce_grid): the values of the 2N grid at the
// points 2r - s (r in Z_N wrapped, s in {0,1}^d given by the bits of `shift`)
// as an N grid, FP64 and FP32 (g: the context's geometry with M = 2N).
ghb_status launch_subgrid(double* out64, float* out32, const double* grid64, const Geometry& g, int shift,
                          cudaStream_t s);
// y = a y + b exp(sign pi i s.m / N) x over a half-spectrum field (m the
// frequency, s the bits of `shift`), skipped when st says the solve is over.
template <typename T>
ghb_status launch_phase(void* y, const void* x, const FieldGeom& fg, int shift, int sign, double a, double b,
                        const CgState* st, cudaStream_t s);
// v *= s for n complex entries
ghb_status launch_scale(double2* v, double s, int64_t n, cudaStream_t st);
// y += a x for n complex entries
ghb_status launch_axpy(double2* y, const double2* x, double a, int64_t n, cudaStream_t st);
// Prolongation of a half-spectrum field from Z_Nc to Z_Nf (Nf_a >= Nc_a, odd):
// the same trigonometric polynomial, coefficients outside Z_Nc zero.
ghb_status launch_prolong(double2* xf, const FieldGeom& ff, const double2* xc, const FieldGeom& fc,
                          cudaStream_t s);
ghb_status launch_add_constant(double2* v, const double2* e, const FieldGeom& fg, const double* E,
                               cudaStream_t s);

// ---------------------------------------------------------------------------
// shared-memory sizing
// ---------------------------------------------------------------------------
// Shared memory of a column tile and the widest tile within ~160 KB (measured:
// 4 FP32 lines of M = 4374 per CTA beat 2 lines at two CTAs per SM by 6-14 %).
__host__ __device__ constexpr size_t col_smem_bytes(int M, int TW, int elem_bytes) {
  return elem_bytes == 8 ? padded_elems<float2>(static_cast<size_t>(M) * TW) * 8
                         : padded_elems<double2>(static_cast<size_t>(M) * TW) * 16;
}
__host__ __device__ constexpr int col_tile_width(int M, int elem_bytes) {
  const size_t budget = 160 * 1024;
  for (int tw : {16, 8, 4, 2}) {
    if (col_smem_bytes(M, tw, elem_bytes) <= budget) return tw;
  }
  return 1;
}

// Transform lengths with size-specialised FP32 and FP64 operator kernels
// (fft_ct.cuh): the double grids 2 * 3^k of the 2-D operator at N = 81, 243,
// 729, 2187, 2187 itself (the reduced operator's transforms at N = 2187), and
// the double grids 72, 135, 270 of the 3-D operator at N = 33, 65, 129.
__host__ __device__ constexpr bool ct_size(int M) {
  return M == 162 || M == 486 || M == 1458 || M == 4374 || M == 2187 || M == 72 || M == 135 || M == 270;
}
template <typename T>
ghb_status launch_col_ct(int sign, int mode, const ColArgs& a, const FftPlan& pl, cudaStream_t s);
template <typename T>
ghb_status launch_row_ct(int NL, const RowArgs& a, const FftPlan& pl, int rows_per_cta, cudaStream_t s);

}  // namespace ghb
