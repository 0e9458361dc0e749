// common.cuh -- internal types and device helpers of the sm_103a state-vector
// library.  Included only by this library's .cu files.
#pragma once

#include <cuda_runtime.h>

#include <complex>
#include <cstdint>
#include <cstdio>
#include <string>
#include <vector>

#include "../../include/qsim.h"

namespace qs {

using cd = std::complex<double>;

// ------------------------------------------------------------------ errors

void set_error(const char* fmt, ...);
int fail(int code, const char* fmt, ...);

#define QS_CUDA(call)                                                                 \
  do {                                                                                \
    cudaError_t e_ = (call);                                                          \
    if (e_ != cudaSuccess)                                                            \
      return ::qs::fail(QS_EDEVICE, "%s: %s (%s:%d)", #call, cudaGetErrorString(e_),  \
                        __FILE__, __LINE__);                                          \
  } while (0)

#define QS_LAUNCHED()                                                                 \
  do {                                                                                \
    cudaError_t e_ = cudaGetLastError();                                              \
    if (e_ != cudaSuccess)                                                            \
      return ::qs::fail(QS_EDEVICE, "kernel launch: %s (%s:%d)", cudaGetErrorString(e_), \
                        __FILE__, __LINE__);                                          \
  } while (0)

#define QS_TRY(expr)              \
  do {                            \
    int rc_ = (expr);             \
    if (rc_ != QS_OK) return rc_; \
  } while (0)

// ------------------------------------------------------------------ index spec
//
// A launch walks "items": item = r * 2^item_log2 + j, register r, local index
// j over the free bits.  The amplitude index of item j inside its register is
// deposit(j): zeros inserted at the fixed bit positions (ascending), then the
// fixed bits' required values OR'ed in.

constexpr int kMaxFix = 48;

struct IdxSpec {
  int nfix;
  int item_log2;              // items per register = 2^item_log2
  uint64_t set_bits;          // required values of the fixed bits
  uint64_t reg_stride;        // amplitudes per register
  uint8_t fix[kMaxFix];       // fixed bit positions, ascending
};

__device__ __forceinline__ uint64_t deposit(uint64_t j, const IdxSpec& s) {
  for (int q = 0; q < s.nfix; ++q) {
    const int p = s.fix[q];
    const uint64_t lo = j & ((1ull << p) - 1ull);
    j = ((j >> p) << (p + 1)) | lo;
  }
  return j | s.set_bits;
}

__device__ __forceinline__ uint64_t item_index(uint64_t item, const IdxSpec& s) {
  const uint64_t r = item >> s.item_log2;
  const uint64_t j = item & ((1ull << s.item_log2) - 1ull);
  return r * s.reg_stride + deposit(j, s);
}

// Builds an IdxSpec over a register of n qubits with the given fixed-bit mask.
int make_idx(int n, uint64_t fixed_mask, uint64_t set_bits, IdxSpec* out);

// ------------------------------------------------------------------ complex math

template <typename R> struct C2;
template <> struct C2<float> { using T = float2; };
template <> struct C2<double> { using T = double2; };

template <typename R> using c2_t = typename C2<R>::T;

template <typename T> __device__ __forceinline__ T cmk(decltype(T::x) a, decltype(T::x) b) {
  T r; r.x = a; r.y = b; return r;
}

// acc + a * b (complex), FMA-contracted
template <typename T> __device__ __forceinline__ T cfma(T a, T b, T acc) {
  acc.x = fma(a.x, b.x, acc.x);
  acc.x = fma(-a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y);
  acc.y = fma(a.y, b.x, acc.y);
  return acc;
}
template <typename T> __device__ __forceinline__ T cmul(T a, T b) {
  T r;
  r.x = fma(a.x, b.x, -a.y * b.y);
  r.y = fma(a.x, b.y, a.y * b.x);
  return r;
}

// two consecutive amplitudes (bit 0 = 0, 1) as one vector access
// ------------------------------------------------------------------ compensated complex64 arithmetic
//
// Knuth's TwoSum (s + e = a + b exactly) and the FMA form of the exact product
// error let a complex64 gate use its FP64 matrix to full accuracy: the matrix
// is held as U_hi + U_lo (both FP32), every output component is summed in
// double-float and rounded to FP32 once.  The _rn intrinsics are never fused
// into FMAs, which the error-free steps rely on.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
__device__ __forceinline__ void cf_first(float& s, float& e, float x, float uh, float ul) {
  s = __fmul_rn(x, uh);
  e = fmaf(x, ul, fmaf(x, uh, -s));
}
__device__ __forceinline__ void cf_add(float& s, float& e, float x, float uh, float ul) {
  const float p = __fmul_rn(x, uh);
  const float pe = fmaf(x, ul, fmaf(x, uh, -p));
  float t, r;
  two_sum(s, p, t, r);
  s = t;
  e = __fadd_rn(e, __fadd_rn(r, pe));
}
// x * u (complex), rounded once
__device__ __forceinline__ float2 cf_mul(float2 x, float2 uh, float2 ul) {
  float rs, re, is, ie;
  cf_first(rs, re, x.x, uh.x, ul.x);
  cf_add(rs, re, -x.y, uh.y, ul.y);
  cf_first(is, ie, x.x, uh.y, ul.y);
  cf_add(is, ie, x.y, uh.x, ul.x);
  return make_float2(__fadd_rn(rs, re), __fadd_rn(is, ie));
}
// u0 * a + u1 * b (complex), rounded once
__device__ __forceinline__ float2 cf_dot2(float2 a, float2 u0h, float2 u0l, float2 b, float2 u1h, float2 u1l) {
  float rs, re, is, ie;
  cf_first(rs, re, a.x, u0h.x, u0l.x);
  cf_add(rs, re, -a.y, u0h.y, u0l.y);
  cf_add(rs, re, b.x, u1h.x, u1l.x);
  cf_add(rs, re, -b.y, u1h.y, u1l.y);
  cf_first(is, ie, a.x, u0h.y, u0l.y);
  cf_add(is, ie, a.y, u0h.x, u0l.x);
  cf_add(is, ie, b.x, u1h.y, u1l.y);
  cf_add(is, ie, b.y, u1h.x, u1l.x);
  return make_float2(__fadd_rn(rs, re), __fadd_rn(is, ie));
}

__device__ __forceinline__ void ld_pair(const float2* p, float2& a0, float2& a1) {
  const float4 v = *reinterpret_cast<const float4*>(p);
  a0 = make_float2(v.x, v.y);
  a1 = make_float2(v.z, v.w);
}
__device__ __forceinline__ void st_pair(float2* p, float2 a0, float2 a1) {
  *reinterpret_cast<float4*>(p) = make_float4(a0.x, a0.y, a1.x, a1.y);
}
__device__ __forceinline__ void ld_pair(const double2* p, double2& a0, double2& a1) {
  a0 = p[0];
  a1 = p[1];
}
__device__ __forceinline__ void st_pair(double2* p, double2 a0, double2 a1) {
  p[0] = a0;
  p[1] = a1;
}

// ------------------------------------------------------------------ host-side objects

struct Workspace {
  void* ptr = nullptr;
  size_t bytes = 0;
};

}  // namespace qs

struct qs_state {
  int dtype = QS_C64;
  int nreg = 0;
  bool uniform = true;               // every register has the same n
  std::vector<int> nq;               // qubits per register
  std::vector<int64_t> off;          // element offsets, nreg + 1
  void* data = nullptr;              // device amplitudes
  size_t bytes = 0;
  bool owns = false;
  cudaStream_t stream = nullptr;
  qs::Workspace ws;                  // reduction scratch, grown on demand
};

struct qs_circuit {
  int nqubits = 0;
  int nparams = 0;
  std::vector<qs_gate_desc> gates;
  std::vector<qs::cd> mats;
  // tile-engine schedule of this circuit (built on first fused apply)
  mutable qs_batch_program* fused = nullptr;
  mutable int fused_tile = 0;
  // k-qubit block plan of this circuit (built on first block apply)
  mutable void* blocks = nullptr;
  mutable int block_k = 0;
  // device tables of the one-launch path (built on first use, rebuilt when the
  // block width, dtype, device or parameters change)
  mutable void* onelaunch = nullptr;
};

struct qs_observable {
  std::vector<qs_pauli_term> terms;
};

namespace qs {

// grow a workspace (stream-ordered free of the old buffer is not needed: we
// synchronise the stream before replacing it)
int ensure_ws(qs_state* s, Workspace& w, size_t bytes);

size_t amp_bytes(int dtype);

// ------------------------------------------------------------------ gate plans

enum OpClass {
  OP_NOP = 0,
  OP_DIAG1,     // amplitude *= (bit t ? d1 : d0) over the fixed-bit subspace (t < 0: d0)
  OP_SWAP1,     // a <-> b (pure X)
  OP_PERM1,     // a' = u01 b, b' = u10 a
  OP_DENSE1,    // [a'; b'] = U [a; b]
  OP_REAL1,     // OP_DENSE1 with a real U (H, Ry): half the multiply-adds
  OP_RXLIKE1,   // OP_DENSE1 with real diagonal, imaginary off-diagonal (Rx): half the multiply-adds
  OP_DIAGK,     // amplitude *= d[m], m = gathered target bits
  OP_PERMK,     // y[m] = v[m] x[perm[m]]
  OP_DENSEK     // y = U x over 2^k tuples
};

struct Plan {
  OpClass op = OP_NOP;
  int k = 0;
  int locs[QS_MAXK] = {0};
  uint64_t ctrl_mask = 0, ctrl_vals = 0;
  // 1-qubit forms
  int t = -1;                       // target (DIAG1: -1 = uniform factor)
  uint64_t mask = 0, vals = 0;      // fixed subspace for DIAG1
  cd d0 = 1, d1 = 1;
  cd u[4];
  bool precise = false;             // complex64: compensated matrix, each output rounded once
  // k-qubit forms (row-major 2^k x 2^k; perm / diag tables)
  std::vector<cd> U;
  int perm[1 << QS_MAXK];
  cd pv[1 << QS_MAXK];
};

// classify a 2^k x 2^k matrix with controls into a kernel plan
int plan_gate(const cd* U, int k, const int* locs, uint64_t ctrl_mask, uint64_t ctrl_vals, Plan* p);

// launch a plan on every register of s (uniform: one launch; uneven: per register)
int launch_plan(qs_state* s, const Plan& p);
// launch a plan on an explicit single-register buffer (used by the adjoint)
int launch_plan_on(void* data, int dtype, int n, int nreg, int64_t reg_stride, const Plan& p,
                   qs_state* owner);

// gate matrices (FP64, row-major), generators and daggers
int named_matrix(int kind, int k, const int32_t* paulis, double theta, std::vector<cd>& U);
int gate_matrix(const qs_circuit* c, const qs_gate_desc& g, const double* params, std::vector<cd>& U);
void dagger(std::vector<cd>& U, int k);
void pauli_string(int k, const int32_t* paulis, std::vector<cd>& S);
int validate_gate(int n, int k, const int32_t* locs, uint64_t ctrl_mask);

// dense 4- and 5-qubit blocks of complex64 states on the tensor cores (tc_block.cu)
void set_tensor_cores(int on);
int tensor_cores_enabled();
bool use_block_tc(int dtype, const Plan& p);
int launch_block_tc(float2* psi, int n, int nreg, const Plan& p, cudaStream_t st);
int tc_status_take();  // QS_ETIMEDOUT (and clears it) if a bounded device wait gave up
int tc_status_address(int** out);  // device address of that status word (current device)
void free_onelaunch(const qs_circuit* c);  // releases the one-launch tables of a circuit
// real Gram matrix sum_x psi_x^T lambda_x of a 4/5-qubit support on the tensor cores
// (interleaved re/im layout), per-CTA partials [grid][W][W]
int gram_tc(int w, const float2* psi, const float2* lam, int n, const int* qubits, double* partials, int* grid_out,
            cudaStream_t st);

// the circuit fused into blocks of at most kmax qubits, gate-by-gate path (blocks.cu)
int apply_blocks(qs_state* s, const qs_circuit* c, const double* params, int kmax, bool precise);
void free_blocks(const qs_circuit* c);

// samples with device uniforms into device indices (reduce.cu)
size_t sample_scratch_doubles(int n);
int sample_dev(const void* data, int dtype, int n, const double* dev_u, int nshots, int64_t* dev_out,
               double* scratch, cudaStream_t st);

// generator H on a gate's targets and c with U = exp(-i theta c H) (adjoint.cu)
int gate_generator(const qs_gate_desc& g, std::vector<cd>& G, double* cfac);
int expect_raw(const void* data, int dtype, int n, int nreg, const qs_observable* o, qs_state* ws_owner,
               double* host_out);

// tile-engine forward of a whole circuit (batch.cu); QS_EUNSUPPORTED if it does not fit
int fused_forward(qs_state* s, const qs_circuit* c, const double* host_params, int tile_qubits);
int fused_backward(qs_state* s, const qs_circuit* c, const double* host_params, const qs_observable* o,
                   void* dev_work, double* host_grad, double* host_loss, int tile_qubits);
void free_fused(qs_batch_program* p);
int schedule_info(const qs_circuit* c, int tile_qubits, int* npasses, int* nphases);
// the scheduler's gate order (expanded SWAPs) and pass of each gate, host only (batch.cu)
int tile_order(const qs_circuit* c, int tile_qubits, std::vector<int>& order, std::vector<int>& pass);

}  // namespace qs
