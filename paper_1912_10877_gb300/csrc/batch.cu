// batch.cu -- batched registers of uneven sizes in one persistent launch
// (Sec. "Batched Quantum Registers"; forward, expectation and reversible
// adjoint of Sec. "Reverse Mode"), complex64.
//
// Every register has its own circuit, parameters and diagonal observable.  The
// host schedules each circuit into fused tile passes (tiles.cuh); a persistent
// grid of 512-thread CTAs takes registers from an atomic counter in
// decreasing-cost order.  A register of n <= 13 qubits lives in shared memory
// for the whole forward, expectation and backward (its lambda too); a larger
// register streams 2^13-amplitude tiles through L2 / HBM once per pass.
// Inside a tile each phase keeps 16 amplitudes per thread in registers.
//
// Backward (Eq. apply-back): the passes and phases run in reverse; for each
// gate, in reverse order, a thread adds Im sum conj(lambda) (G psi) over its
// pairs (FP32 over <= 8 pairs, then FP32 warp shuffles, FP64 from the warp
// level up) and uncomputes psi and lambda with U^dagger in FP32, using the
// structured Rx / Ry / diagonal forms of the inverse rotations.  The
// register's gradient lives in shared memory (FP64) and is written once.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>

#include "tiles.cuh"

namespace qs {

constexpr int kMaxRegParams = 2048;
constexpr int kMaxPhaseOps = 64;
constexpr int kBatchTile = kMaxTileBits;

struct GSpec {           // one circuit gate of one register
  int32_t kind;
  int32_t param;         // global index into params (-1: theta)
  double theta;
  double2 mat[4];        // MATRIX gates (1 target)
};

struct FMem {            // members of a fused forward op (applied in order)
  int32_t count;
  int32_t g[4];          // global GSpec indices
};

struct BReg {
  int32_t n, m, npass, pass0;
  int32_t nparam, nterm, term0, pad;
  int64_t amp_off;       // elements into the batch state
  int64_t work_off;      // elements into psi/lambda work buffers (n > 13), -1 otherwise
  int64_t param_off;     // into params / grad
  double cost;
};

struct BTerm {
  double coeff;
  uint64_t z;
};

struct BArgs {
  float2* state;
  float2* wpsi;          // backward work copies of psi (registers larger than the tile)
  float2* wlam;          // lambda (same)
  float4* wpsif;         // precise path: double-float psi work copies
  float4* wlamf;         // precise path: double-float lambda
  const float2* flo;     // precise path: corrections U - U_hi of the forward ops (4 each)
  const float2* dtlo;    // precise path: corrections of the diagonal tables (16 each)
  const float2* blo;     // precise path: corrections of the backward ops' U^dagger (4 each)
  const BReg* regs;
  const int32_t* order;
  const TPass* passes;
  const TPhase* phases;
  const TOp* fops;
  const TOp* bops;
  const float2* dtab;    // TK_DIAG16 factor tables
  const DRun* druns;     // TK_DIAGRUN entries
  const BTerm* terms;
  double* loss;
  double* grad;
  int* counter;
  int nreg;
  int flags;
};

enum { BF_RESET = 1, BF_GRAD = 2 };

// ------------------------------------------------------------------ device: ops on the amplitudes of a phase
//
// A phase of RB register bits (RB = 2..4) keeps 2^RB amplitudes per thread in
// registers.  The complex64 path computes in FP32.  The precise path of the
// batched engine (PREC) applies the forward gates with compensated matrices
// (every FP32 entry U_hi has a correction U_lo = U - U_hi kept beside it, so
// the state sees U to ~2^-48 while it is still stored and multiplied in FP32)
// and runs the reversible uncompute of psi and lambda in double-float
// arithmetic (each real number a pair hi + lo of FP32 values, ~48 bits): the
// uncompute is FP64-class without the FP64 units, which run at 1/64 of the
// FP32 rate on this GPU.

__device__ __forceinline__ float2 cmulf(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 cmaf(float2 a, float2 b, float2 c) {  // a*b + c
  c.x = fmaf(a.x, b.x, c.x);
  c.x = fmaf(-a.y, b.y, c.x);
  c.y = fmaf(a.x, b.y, c.y);
  c.y = fmaf(a.y, b.x, c.y);
  return c;
}
__device__ __forceinline__ float imcj(float2 p, float2 q) { return fmaf(p.x, q.y, -p.y * q.x); }  // Im(conj(p) q)
__device__ __forceinline__ float recj(float2 p, float2 q) { return fmaf(p.x, q.x, p.y * q.y); }   // Re(conj(p) q)

// (a, b) <- U (a, b) for the structured kinds; U row-major in u0..u3
// a diagonal whose first entry is exactly 1 (shift, controlled phases): only b changes
constexpr int TK_DIAGB = 16;

template <int KIND>
__device__ __forceinline__ void pair_apply(float2& a, float2& b, float2 u0, float2 u1, float2 u2, float2 u3) {
  if (KIND == TK_SWAP) {
    const float2 t = a; a = b; b = t;
  } else if (KIND == TK_DIAGB) {
    b = cmulf(b, u3);
  } else if (KIND == TK_DIAG) {
    a = cmulf(a, u0);
    b = cmulf(b, u3);
  } else if (KIND == TK_RX) {  // [[c, i s], [i s, c]] (c = u0.x, s = u1.y)
    const float c = u0.x, s = u1.y;
    const float2 na = make_float2(fmaf(c, a.x, -s * b.y), fmaf(c, a.y, s * b.x));
    const float2 nb = make_float2(fmaf(c, b.x, -s * a.y), fmaf(c, b.y, s * a.x));
    a = na; b = nb;
  } else if (KIND == TK_RY) {  // real [[c, u1], [u2, c]]
    const float c = u0.x, p = u1.x, q = u2.x;
    const float2 na = make_float2(fmaf(c, a.x, p * b.x), fmaf(c, a.y, p * b.y));
    const float2 nb = make_float2(fmaf(q, a.x, c * b.x), fmaf(q, a.y, c * b.y));
    a = na; b = nb;
  } else {
    const float2 na = cmaf(u1, b, cmulf(u0, a));
    const float2 nb = cmaf(u3, b, cmulf(u2, a));
    a = na; b = nb;
  }
}

// compensated forward (cf_mul / cf_dot2: the FP64-exact matrix applied to the
// FP32 amplitudes in double-float, each output rounded to FP32 once)
template <int KIND>
__device__ __forceinline__ void pair_apply_c(float2& a, float2& b, const float2 (&u)[4], const float2 (&w)[4]) {
  if (KIND == TK_SWAP) {
    const float2 t = a; a = b; b = t;
  } else if (KIND == TK_DIAG) {
    a = cf_mul(a, u[0], w[0]);
    b = cf_mul(b, u[3], w[3]);
  } else {
    const float2 na = cf_dot2(a, u[0], w[0], b, u[1], w[1]);
    const float2 nb = cf_dot2(a, u[2], w[2], b, u[3], w[3]);
    a = na; b = nb;
  }
}

template <int RB, int T, int KIND, bool CTRL>
__device__ __forceinline__ void op_fwd(float2 (&x)[1 << RB], const TOp& op) {
  const int cm = op.cmask, cv = op.cval;
  const float2 u0 = op.u[0], u1 = op.u[1], u2 = op.u[2], u3 = op.u[3];
#pragma unroll
  for (int j = 0; j < (1 << RB); ++j) {
    if (j & (1 << T)) continue;
    if (CTRL && (j & cm) != cv) continue;
    pair_apply<KIND>(x[j], x[j | (1 << T)], u0, u1, u2, u3);
  }
}

template <int RB, int T, int KIND, bool CTRL>
__device__ __forceinline__ void op_fwd_c(float2 (&x)[1 << RB], const TOp& op, const float2* lo) {
  const int cm = op.cmask, cv = op.cval;
  const float2 u[4] = {op.u[0], op.u[1], op.u[2], op.u[3]};
  const float2 w[4] = {lo[0], lo[1], lo[2], lo[3]};
#pragma unroll
  for (int j = 0; j < (1 << RB); ++j) {
    if (j & (1 << T)) continue;
    if (CTRL && (j & cm) != cv) continue;
    pair_apply_c<KIND>(x[j], x[j | (1 << T)], u, w);
  }
}

template <int RB, int T, bool COMP>
__device__ __forceinline__ void op_fwd_k(float2 (&x)[1 << RB], const TOp& op, const float2* lo) {
  if (COMP) {
    if (op.kind == TK_SWAP) op_fwd<RB, T, TK_SWAP, true>(x, op);
    else if (op.cmask == 0) {
      if (op.kind == TK_DIAG) op_fwd_c<RB, T, TK_DIAG, false>(x, op, lo);
      else op_fwd_c<RB, T, TK_DENSE, false>(x, op, lo);
    } else {
      if (op.kind == TK_DIAG) op_fwd_c<RB, T, TK_DIAG, true>(x, op, lo);
      else op_fwd_c<RB, T, TK_DENSE, true>(x, op, lo);
    }
    return;
  }
  const bool one0 = op.u[0].x == 1.f && op.u[0].y == 0.f;  // uniform across the CTA
  if (op.kind == TK_SWAP) op_fwd<RB, T, TK_SWAP, true>(x, op);
  else if (op.cmask == 0) {
    if (op.kind == TK_DIAG) {
      if (one0) op_fwd<RB, T, TK_DIAGB, false>(x, op);
      else op_fwd<RB, T, TK_DIAG, false>(x, op);
    } else {
      op_fwd<RB, T, TK_DENSE, false>(x, op);
    }
  } else {
    if (op.kind == TK_DIAG) {
      if (one0) op_fwd<RB, T, TK_DIAGB, true>(x, op);
      else op_fwd<RB, T, TK_DIAG, true>(x, op);
    } else {
      op_fwd<RB, T, TK_DENSE, true>(x, op);
    }
  }
}

// x_j *= (bit T of j ? p1 : p0)
template <int RB, int T>
__device__ __forceinline__ void mul_by_bit(float2 (&x)[1 << RB], float2 p0, float2 p1) {
#pragma unroll
  for (int j = 0; j < (1 << RB); ++j) x[j] = cmulf(x[j], ((j >> T) & 1) ? p1 : p0);
}

// a TK_DIAGRUN op: the products p0, p1 of its entries' factors where their
// controls hold (selects, no branch on the thread's bits), then one pass over
// the amplitudes by phase bit t
template <int RB>
__device__ __forceinline__ void diag_run(float2 (&x)[1 << RB], const TOp& op, const DRun* runs, uint32_t gb) {
  float2 p0 = make_float2(1.f, 0.f), p1 = p0;
  const DRun* e = runs + op.param;
#pragma unroll 2
  for (uint32_t k = 0; k < op.count; ++k) {
    const uint4* w = reinterpret_cast<const uint4*>(e + k);
    const uint4 a = w[0], b = w[1];  // tmask, tval, gate, tq | u0, u3
    const float2 u0 = make_float2(__uint_as_float(b.x), __uint_as_float(b.y));
    const float2 u3 = make_float2(__uint_as_float(b.z), __uint_as_float(b.w));
    const bool on = (gb & a.x) == a.y;
    float2 f0 = u0, f1 = u3;
    if (a.w != 0xffffffffu) {  // target outside the phase: one factor by its bit
      f0 = ((gb >> (a.w & 31u)) & 1u) ? u3 : u0;
      f1 = f0;
    }
    const float2 q0 = cmulf(p0, f0), q1 = cmulf(p1, f1);
    p0 = on ? q0 : p0;
    p1 = on ? q1 : p1;
  }
  switch (op.t) {
    case 0: mul_by_bit<RB, 0>(x, p0, p1); break;
    case 1: mul_by_bit<RB, 1>(x, p0, p1); break;
    case 2: if constexpr (RB > 2) mul_by_bit<RB, 2>(x, p0, p1); break;
    default: if constexpr (RB > 3) mul_by_bit<RB, 3>(x, p0, p1); break;
  }
}

// Forward op forms by TOp::var: 0 out-of-phase diagonal, 1 diagonal table,
// 2 + t controlled swap, 6 + t / 10 + t diagonal without / with phase-local
// controls, 14 + t / 18 + t dense without / with them (t: target phase bit),
// 22 a run of diagonal gates (TK_DIAGRUN)
enum { FV_DIAGOUT = 0, FV_DIAG16 = 1, FV_SWAP = 2, FV_DIAG = 6, FV_DIAGC = 10, FV_DENSE = 14, FV_DENSEC = 18,
       FV_DIAGRUN = 22 };

template <int RB, int T, int KIND, bool CTRL, bool COMP>
__device__ __forceinline__ void fwd_form(float2 (&x)[1 << RB], const TOp& op, const float2* lo) {
  if constexpr (T < RB) {
    if constexpr (KIND == TK_SWAP) {
      op_fwd<RB, T, TK_SWAP, true>(x, op);
    } else if constexpr (COMP) {
      op_fwd_c<RB, T, KIND, CTRL>(x, op, lo);
    } else if constexpr (KIND == TK_DIAG) {
      if (op.u[0].x == 1.f && op.u[0].y == 0.f) op_fwd<RB, T, TK_DIAGB, CTRL>(x, op);
      else op_fwd<RB, T, TK_DIAG, CTRL>(x, op);
    } else {
      op_fwd<RB, T, KIND, CTRL>(x, op);
    }
  }
}

template <int RB, bool COMP>
__device__ __forceinline__ void apply_fwd_var(float2 (&x)[1 << RB], const TOp& op, const float2* lo,
                                              const DRun* runs, uint32_t gb) {
  switch (op.var) {
    case FV_DIAGRUN:
      if constexpr (!COMP) diag_run<RB>(x, op, runs, gb);
      break;
    case FV_SWAP + 0: fwd_form<RB, 0, TK_SWAP, true, COMP>(x, op, lo); break;
    case FV_SWAP + 1: fwd_form<RB, 1, TK_SWAP, true, COMP>(x, op, lo); break;
    case FV_SWAP + 2: fwd_form<RB, 2, TK_SWAP, true, COMP>(x, op, lo); break;
    case FV_SWAP + 3: fwd_form<RB, 3, TK_SWAP, true, COMP>(x, op, lo); break;
    case FV_DIAG + 0: fwd_form<RB, 0, TK_DIAG, false, COMP>(x, op, lo); break;
    case FV_DIAG + 1: fwd_form<RB, 1, TK_DIAG, false, COMP>(x, op, lo); break;
    case FV_DIAG + 2: fwd_form<RB, 2, TK_DIAG, false, COMP>(x, op, lo); break;
    case FV_DIAG + 3: fwd_form<RB, 3, TK_DIAG, false, COMP>(x, op, lo); break;
    case FV_DIAGC + 0: fwd_form<RB, 0, TK_DIAG, true, COMP>(x, op, lo); break;
    case FV_DIAGC + 1: fwd_form<RB, 1, TK_DIAG, true, COMP>(x, op, lo); break;
    case FV_DIAGC + 2: fwd_form<RB, 2, TK_DIAG, true, COMP>(x, op, lo); break;
    case FV_DIAGC + 3: fwd_form<RB, 3, TK_DIAG, true, COMP>(x, op, lo); break;
    case FV_DENSE + 0: fwd_form<RB, 0, TK_DENSE, false, COMP>(x, op, lo); break;
    case FV_DENSE + 1: fwd_form<RB, 1, TK_DENSE, false, COMP>(x, op, lo); break;
    case FV_DENSE + 2: fwd_form<RB, 2, TK_DENSE, false, COMP>(x, op, lo); break;
    case FV_DENSE + 3: fwd_form<RB, 3, TK_DENSE, false, COMP>(x, op, lo); break;
    case FV_DENSEC + 0: fwd_form<RB, 0, TK_DENSE, true, COMP>(x, op, lo); break;
    case FV_DENSEC + 1: fwd_form<RB, 1, TK_DENSE, true, COMP>(x, op, lo); break;
    case FV_DENSEC + 2: fwd_form<RB, 2, TK_DENSE, true, COMP>(x, op, lo); break;
    case FV_DENSEC + 3: fwd_form<RB, 3, TK_DENSE, true, COMP>(x, op, lo); break;
    default: break;
  }
}

template <int RB, bool COMP>
__device__ __forceinline__ void apply_fwd(float2 (&x)[1 << RB], const TOp& op, const float2* lo) {
  switch (op.t) {
    case 0: op_fwd_k<RB, 0, COMP>(x, op, lo); break;
    case 1: op_fwd_k<RB, 1, COMP>(x, op, lo); break;
    case 2: if constexpr (RB > 2) op_fwd_k<RB, 2, COMP>(x, op, lo); break;
    default: if constexpr (RB > 3) op_fwd_k<RB, 3, COMP>(x, op, lo); break;
  }
}

// Backward op: first this thread's share of Im<lambda|G|psi> over its pairs
// (GK 0: none; 1: diagonal generator diag(g0, g3); 2: X; 3: Y), then
// psi <- U^dag psi and lambda <- U^dag lambda.
template <int RB, int T, int KIND, int GK, bool CTRL>
__device__ __forceinline__ float op_bwd(float2 (&x)[1 << RB], float2 (&l)[1 << RB], const TOp& op, float g0, float g3) {
  const int cm = op.cmask, cv = op.cval;
  const float2 u0 = op.u[0], u1 = op.u[1], u2 = op.u[2], u3 = op.u[3];
  float acc = 0.f;
#pragma unroll
  for (int j = 0; j < (1 << RB); ++j) {
    if (j & (1 << T)) continue;
    if (CTRL && (j & cm) != cv) continue;
    const int k = j | (1 << T);
    if (GK == 1) acc += fmaf(g0, imcj(l[j], x[j]), g3 * imcj(l[k], x[k]));
    if (GK == 2) acc += imcj(l[j], x[k]) + imcj(l[k], x[j]);
    if (GK == 3) acc += recj(l[k], x[j]) - recj(l[j], x[k]);
    pair_apply<KIND>(x[j], x[k], u0, u1, u2, u3);
    pair_apply<KIND>(l[j], l[k], u0, u1, u2, u3);
  }
  return acc;
}

template <int RB, int T, bool CTRL>
__device__ __forceinline__ float op_bwd_c(float2 (&x)[1 << RB], float2 (&l)[1 << RB], const TOp& op) {
  switch (op.gen) {
    case GEN_X: return op_bwd<RB, T, TK_RX, 2, CTRL>(x, l, op, 0.f, 0.f);
    case GEN_Y: return op_bwd<RB, T, TK_RY, 3, CTRL>(x, l, op, 0.f, 0.f);
    case GEN_Z: return op_bwd<RB, T, TK_DIAG, 1, CTRL>(x, l, op, 1.f, -1.f);
    case GEN_P1: return op_bwd<RB, T, TK_DIAG, 1, CTRL>(x, l, op, 0.f, 1.f);
    default: return op_bwd<RB, T, TK_DIAG, 1, CTRL>(x, l, op, 1.f, 1.f);  // GEN_I
  }
}

template <int RB, int T>
__device__ __forceinline__ float op_bwd_t(float2 (&x)[1 << RB], float2 (&l)[1 << RB], const TOp& op) {
  if (op.gen == GEN_NONE) {
    if (op.kind == TK_SWAP) return op_bwd<RB, T, TK_SWAP, 0, true>(x, l, op, 0.f, 0.f);
    if (op.kind == TK_DIAG) return op_bwd<RB, T, TK_DIAG, 0, true>(x, l, op, 0.f, 0.f);
    return op_bwd<RB, T, TK_DENSE, 0, true>(x, l, op, 0.f, 0.f);
  }
  return op.cmask ? op_bwd_c<RB, T, true>(x, l, op) : op_bwd_c<RB, T, false>(x, l, op);
}

// backward op forms (TOp::var = 13 t + form): 0 controlled swap, 1 / 2 diagonal /
// dense without a parameter, then X, Y, Z, P1, I generators, each without and
// with phase-local controls
template <int RB, int T, int F>
__device__ __forceinline__ float bwd_form(float2 (&x)[1 << RB], float2 (&l)[1 << RB], const TOp& op) {
  if constexpr (T >= RB) {
    return 0.f;
  } else if constexpr (F == 0) {
    return op_bwd<RB, T, TK_SWAP, 0, true>(x, l, op, 0.f, 0.f);
  } else if constexpr (F == 1) {
    return op_bwd<RB, T, TK_DIAG, 0, true>(x, l, op, 0.f, 0.f);
  } else if constexpr (F == 2) {
    return op_bwd<RB, T, TK_DENSE, 0, true>(x, l, op, 0.f, 0.f);
  } else {
    constexpr bool C = ((F - 3) & 1) != 0;
    constexpr int G = (F - 3) / 2;
    if constexpr (G == 0) return op_bwd<RB, T, TK_RX, 2, C>(x, l, op, 0.f, 0.f);
    else if constexpr (G == 1) return op_bwd<RB, T, TK_RY, 3, C>(x, l, op, 0.f, 0.f);
    else if constexpr (G == 2) return op_bwd<RB, T, TK_DIAG, 1, C>(x, l, op, 1.f, -1.f);
    else if constexpr (G == 3) return op_bwd<RB, T, TK_DIAG, 1, C>(x, l, op, 0.f, 1.f);
    else return op_bwd<RB, T, TK_DIAG, 1, C>(x, l, op, 1.f, 1.f);
  }
}

template <int RB>
__device__ __forceinline__ float apply_bwd_var(float2 (&x)[1 << RB], float2 (&l)[1 << RB], const TOp& op) {
  switch (op.var) {
    case 0: return bwd_form<RB, 0, 0>(x, l, op);
    case 1: return bwd_form<RB, 0, 1>(x, l, op);
    case 2: return bwd_form<RB, 0, 2>(x, l, op);
    case 3: return bwd_form<RB, 0, 3>(x, l, op);
    case 4: return bwd_form<RB, 0, 4>(x, l, op);
    case 5: return bwd_form<RB, 0, 5>(x, l, op);
    case 6: return bwd_form<RB, 0, 6>(x, l, op);
    case 7: return bwd_form<RB, 0, 7>(x, l, op);
    case 8: return bwd_form<RB, 0, 8>(x, l, op);
    case 9: return bwd_form<RB, 0, 9>(x, l, op);
    case 10: return bwd_form<RB, 0, 10>(x, l, op);
    case 11: return bwd_form<RB, 0, 11>(x, l, op);
    case 12: return bwd_form<RB, 0, 12>(x, l, op);
    case 13: return bwd_form<RB, 1, 0>(x, l, op);
    case 14: return bwd_form<RB, 1, 1>(x, l, op);
    case 15: return bwd_form<RB, 1, 2>(x, l, op);
    case 16: return bwd_form<RB, 1, 3>(x, l, op);
    case 17: return bwd_form<RB, 1, 4>(x, l, op);
    case 18: return bwd_form<RB, 1, 5>(x, l, op);
    case 19: return bwd_form<RB, 1, 6>(x, l, op);
    case 20: return bwd_form<RB, 1, 7>(x, l, op);
    case 21: return bwd_form<RB, 1, 8>(x, l, op);
    case 22: return bwd_form<RB, 1, 9>(x, l, op);
    case 23: return bwd_form<RB, 1, 10>(x, l, op);
    case 24: return bwd_form<RB, 1, 11>(x, l, op);
    case 25: return bwd_form<RB, 1, 12>(x, l, op);
    case 26: return bwd_form<RB, 2, 0>(x, l, op);
    case 27: return bwd_form<RB, 2, 1>(x, l, op);
    case 28: return bwd_form<RB, 2, 2>(x, l, op);
    case 29: return bwd_form<RB, 2, 3>(x, l, op);
    case 30: return bwd_form<RB, 2, 4>(x, l, op);
    case 31: return bwd_form<RB, 2, 5>(x, l, op);
    case 32: return bwd_form<RB, 2, 6>(x, l, op);
    case 33: return bwd_form<RB, 2, 7>(x, l, op);
    case 34: return bwd_form<RB, 2, 8>(x, l, op);
    case 35: return bwd_form<RB, 2, 9>(x, l, op);
    case 36: return bwd_form<RB, 2, 10>(x, l, op);
    case 37: return bwd_form<RB, 2, 11>(x, l, op);
    case 38: return bwd_form<RB, 2, 12>(x, l, op);
    case 39: return bwd_form<RB, 3, 0>(x, l, op);
    case 40: return bwd_form<RB, 3, 1>(x, l, op);
    case 41: return bwd_form<RB, 3, 2>(x, l, op);
    case 42: return bwd_form<RB, 3, 3>(x, l, op);
    case 43: return bwd_form<RB, 3, 4>(x, l, op);
    case 44: return bwd_form<RB, 3, 5>(x, l, op);
    case 45: return bwd_form<RB, 3, 6>(x, l, op);
    case 46: return bwd_form<RB, 3, 7>(x, l, op);
    case 47: return bwd_form<RB, 3, 8>(x, l, op);
    case 48: return bwd_form<RB, 3, 9>(x, l, op);
    case 49: return bwd_form<RB, 3, 10>(x, l, op);
    case 50: return bwd_form<RB, 3, 11>(x, l, op);
    case 51: return bwd_form<RB, 3, 12>(x, l, op);
    default: return 0.f;
  }
}

template <int RB>
__device__ __forceinline__ float apply_bwd(float2 (&x)[1 << RB], float2 (&l)[1 << RB], const TOp& op) {
  switch (op.t) {
    case 0: return op_bwd_t<RB, 0>(x, l, op);
    case 1: return op_bwd_t<RB, 1>(x, l, op);
    case 2: if constexpr (RB > 2) return op_bwd_t<RB, 2>(x, l, op); return 0.f;
    default: if constexpr (RB > 3) return op_bwd_t<RB, 3>(x, l, op); return 0.f;
  }
}

// ------------------------------------------------------------------ device: double-float arithmetic
//
// A double-float value is an unevaluated sum hi + lo of two FP32 numbers with
// |lo| <= ulp(hi) / 2 (Dekker 1971).  The building blocks are Knuth's
// error-free TwoSum and the FMA form of TwoProduct (the rounding error of
// a * b is fma(a, b, -a * b) exactly); a sum of products accumulates the large
// parts with TwoSum and every small part in a running FP32 correction, and is
// renormalised once at the end (Joldes, Muller and Popescu, ACM TOMS 2017,
// give the error bounds of these double-word operations).  The _rn
// intrinsics keep the compiler from fusing the exact-error steps.

struct ffc {         // complex double-float: (h.x + l.x) + i (h.y + l.y)
  float2 h, l;
};


struct DWAcc {       // running sum s + e of double-float products
  float s, e;
};

// (xh + xl) * (yh + yl) without the xl * yl term (below 2^-48 relative)
__device__ __forceinline__ void dw_first(DWAcc& A, float xh, float xl, float yh, float yl) {
  A.s = __fmul_rn(xh, yh);
  A.e = fmaf(xh, yl, fmaf(xl, yh, fmaf(xh, yh, -A.s)));
}
__device__ __forceinline__ void dw_add(DWAcc& A, float xh, float xl, float yh, float yl) {
  const float p = __fmul_rn(xh, yh);
  const float pe = fmaf(xh, yl, fmaf(xl, yh, fmaf(xh, yh, -p)));
  float s, t;
  two_sum(A.s, p, s, t);
  A.s = s;
  A.e = __fadd_rn(A.e, __fadd_rn(t, pe));
}
__device__ __forceinline__ void dw_out(const DWAcc& A, float& h, float& l) { two_sum(A.s, A.e, h, l); }

// a * u for complex double-floats (u = uh + ul)
__device__ __forceinline__ ffc ff_cmul(const ffc& a, float2 uh, float2 ul) {
  DWAcc re, im;
  dw_first(re, a.h.x, a.l.x, uh.x, ul.x);
  dw_add(re, -a.h.y, -a.l.y, uh.y, ul.y);
  dw_first(im, a.h.x, a.l.x, uh.y, ul.y);
  dw_add(im, a.h.y, a.l.y, uh.x, ul.x);
  ffc r;
  dw_out(re, r.h.x, r.l.x);
  dw_out(im, r.h.y, r.l.y);
  return r;
}

// u0 * a + u1 * b for complex double-floats
__device__ __forceinline__ ffc ff_cdot2(const ffc& a, float2 u0h, float2 u0l, const ffc& b, float2 u1h, float2 u1l) {
  DWAcc re, im;
  dw_first(re, a.h.x, a.l.x, u0h.x, u0l.x);
  dw_add(re, -a.h.y, -a.l.y, u0h.y, u0l.y);
  dw_add(re, b.h.x, b.l.x, u1h.x, u1l.x);
  dw_add(re, -b.h.y, -b.l.y, u1h.y, u1l.y);
  dw_first(im, a.h.x, a.l.x, u0h.y, u0l.y);
  dw_add(im, a.h.y, a.l.y, u0h.x, u0l.x);
  dw_add(im, b.h.x, b.l.x, u1h.y, u1l.y);
  dw_add(im, b.h.y, b.l.y, u1h.x, u1l.x);
  ffc r;
  dw_out(re, r.h.x, r.l.x);
  dw_out(im, r.h.y, r.l.y);
  return r;
}

// (a, b) <- U (a, b) in double-float; U = u + w (hi + lo), row-major
template <int KIND>
__device__ __forceinline__ void pair_apply_ff(ffc& a, ffc& b, const float2 (&u)[4], const float2 (&w)[4]) {
  if (KIND == TK_SWAP) {
    const ffc t = a; a = b; b = t;
  } else if (KIND == TK_DIAG) {
    a = ff_cmul(a, u[0], w[0]);
    b = ff_cmul(b, u[3], w[3]);
  } else if (KIND == TK_RX) {  // [[c, i s], [i s, c]]: a' = c a + i s b
    const float ch = u[0].x, cl = w[0].x, sh = u[1].y, sl = w[1].y;
    DWAcc r0, i0, r1, i1;
    dw_first(r0, a.h.x, a.l.x, ch, cl); dw_add(r0, -b.h.y, -b.l.y, sh, sl);
    dw_first(i0, a.h.y, a.l.y, ch, cl); dw_add(i0, b.h.x, b.l.x, sh, sl);
    dw_first(r1, b.h.x, b.l.x, ch, cl); dw_add(r1, -a.h.y, -a.l.y, sh, sl);
    dw_first(i1, b.h.y, b.l.y, ch, cl); dw_add(i1, a.h.x, a.l.x, sh, sl);
    dw_out(r0, a.h.x, a.l.x); dw_out(i0, a.h.y, a.l.y);
    dw_out(r1, b.h.x, b.l.x); dw_out(i1, b.h.y, b.l.y);
  } else if (KIND == TK_RY) {  // real [[c, p], [q, c]]
    const float ch = u[0].x, cl = w[0].x, ph = u[1].x, pl = w[1].x, qh = u[2].x, ql = w[2].x;
    DWAcc r0, i0, r1, i1;
    dw_first(r0, a.h.x, a.l.x, ch, cl); dw_add(r0, b.h.x, b.l.x, ph, pl);
    dw_first(i0, a.h.y, a.l.y, ch, cl); dw_add(i0, b.h.y, b.l.y, ph, pl);
    dw_first(r1, a.h.x, a.l.x, qh, ql); dw_add(r1, b.h.x, b.l.x, ch, cl);
    dw_first(i1, a.h.y, a.l.y, qh, ql); dw_add(i1, b.h.y, b.l.y, ch, cl);
    dw_out(r0, a.h.x, a.l.x); dw_out(i0, a.h.y, a.l.y);
    dw_out(r1, b.h.x, b.l.x); dw_out(i1, b.h.y, b.l.y);
  } else {
    const ffc na = ff_cdot2(a, u[0], w[0], b, u[1], w[1]);
    const ffc nb = ff_cdot2(a, u[2], w[2], b, u[3], w[3]);
    a = na; b = nb;
  }
}

// the backward op of the precise path: gradient share from the hi parts
// (FP32 products, FP64 above the warp), then the double-float uncompute
template <int RB, int T, int KIND, int GK, bool CTRL>
__device__ __forceinline__ float op_bwd_ff(ffc (&x)[1 << RB], ffc (&l)[1 << RB], const TOp& op, const float2* lo,
                                           float g0, float g3) {
  const int cm = op.cmask, cv = op.cval;
  const float2 u[4] = {op.u[0], op.u[1], op.u[2], op.u[3]};
  const float2 w[4] = {lo[0], lo[1], lo[2], lo[3]};
  float acc = 0.f;
#pragma unroll
  for (int j = 0; j < (1 << RB); ++j) {
    if (j & (1 << T)) continue;
    if (CTRL && (j & cm) != cv) continue;
    const int k = j | (1 << T);
    if (GK == 1) acc += fmaf(g0, imcj(l[j].h, x[j].h), g3 * imcj(l[k].h, x[k].h));
    if (GK == 2) acc += imcj(l[j].h, x[k].h) + imcj(l[k].h, x[j].h);
    if (GK == 3) acc += recj(l[k].h, x[j].h) - recj(l[j].h, x[k].h);
    pair_apply_ff<KIND>(x[j], x[k], u, w);
    pair_apply_ff<KIND>(l[j], l[k], u, w);
  }
  return acc;
}

template <int RB, int T, bool CTRL>
__device__ __forceinline__ float op_bwd_ff_c(ffc (&x)[1 << RB], ffc (&l)[1 << RB], const TOp& op, const float2* lo) {
  switch (op.gen) {
    case GEN_X: return op_bwd_ff<RB, T, TK_RX, 2, CTRL>(x, l, op, lo, 0.f, 0.f);
    case GEN_Y: return op_bwd_ff<RB, T, TK_RY, 3, CTRL>(x, l, op, lo, 0.f, 0.f);
    case GEN_Z: return op_bwd_ff<RB, T, TK_DIAG, 1, CTRL>(x, l, op, lo, 1.f, -1.f);
    case GEN_P1: return op_bwd_ff<RB, T, TK_DIAG, 1, CTRL>(x, l, op, lo, 0.f, 1.f);
    default: return op_bwd_ff<RB, T, TK_DIAG, 1, CTRL>(x, l, op, lo, 1.f, 1.f);  // GEN_I
  }
}

template <int RB, int T>
__device__ __forceinline__ float op_bwd_ff_t(ffc (&x)[1 << RB], ffc (&l)[1 << RB], const TOp& op, const float2* lo) {
  if (op.gen == GEN_NONE) {
    if (op.kind == TK_SWAP) return op_bwd_ff<RB, T, TK_SWAP, 0, true>(x, l, op, lo, 0.f, 0.f);
    if (op.kind == TK_DIAG) return op_bwd_ff<RB, T, TK_DIAG, 0, true>(x, l, op, lo, 0.f, 0.f);
    return op_bwd_ff<RB, T, TK_DENSE, 0, true>(x, l, op, lo, 0.f, 0.f);
  }
  return op.cmask ? op_bwd_ff_c<RB, T, true>(x, l, op, lo) : op_bwd_ff_c<RB, T, false>(x, l, op, lo);
}

template <int RB>
__device__ __forceinline__ float apply_bwd_ff(ffc (&x)[1 << RB], ffc (&l)[1 << RB], const TOp& op, const float2* lo) {
  switch (op.t) {
    case 0: return op_bwd_ff_t<RB, 0>(x, l, op, lo);
    case 1: return op_bwd_ff_t<RB, 1>(x, l, op, lo);
    case 2: if constexpr (RB > 2) return op_bwd_ff_t<RB, 2>(x, l, op, lo); return 0.f;
    default: if constexpr (RB > 3) return op_bwd_ff_t<RB, 3>(x, l, op, lo); return 0.f;
  }
}

// ------------------------------------------------------------------ device: the persistent kernel

constexpr int kWarps = kTileThreads / 32;

struct BShared {
  double grad[kMaxRegParams];
  float red[kMaxPhaseOps * kWarps];
  double lred[kWarps];
  uint32_t rowoff[1 << (kMaxTileBits - kRowBits)];  // register offset of each 32-amplitude tile row (current pass)
  int reg;
};

// Tile rows: tile-local bits 0..4 are register qubits 0..4 (planner seed), so a
// row of 32 amplitudes is contiguous (256 bytes).  rowoff[] holds the register
// offset of every row of the current pass; tile_base() the offset of a tile.
__device__ void set_rows(uint32_t* rowoff, const TPass& p, int m) {
  for (uint32_t row = threadIdx.x; row < (1u << (m - kRowBits)); row += blockDim.x) {
    uint32_t o = 0;
    for (int k = kRowBits; k < m; ++k) o |= ((row >> (k - kRowBits)) & 1u) << p.tbits[k];
    rowoff[row] = o;
  }
  __syncthreads();
}

__device__ __forceinline__ uint64_t tile_base(uint64_t tile, const TPass& p, int g) {
  uint64_t o = 0;
  for (int k = 0; k < g; ++k) o |= ((tile >> k) & 1ull) << p.gbits[k];
  return o;
}

// Stage one or two tiles (2^m amplitudes each) between global and shared
// memory.  Each thread issues up to 8 16-byte loads per tile before any shared
// store (4096 loads of one tile in flight per CTA).
constexpr int kLdChunk = 8;

template <bool TWO>
__device__ __noinline__ void load_tiles(float2* sm0, const float2* src0, float2* sm1, const float2* src1,
                                        const uint32_t* rowoff, int m) {
  const uint32_t nq = 1u << (m - 1);  // float4 per tile
  constexpr int C = TWO ? kLdChunk / 2 : kLdChunk;
  for (uint32_t q0 = 0; q0 < nq; q0 += C * kTileThreads) {
    float4 v0[C], v1[C];
#pragma unroll
    for (int k = 0; k < C; ++k) {
      const uint32_t q = q0 + threadIdx.x + k * kTileThreads;
      if (q < nq) {
        const uint32_t off = rowoff[q >> 4] + 2 * (q & 15);
        v0[k] = *reinterpret_cast<const float4*>(src0 + off);
        if (TWO) v1[k] = *reinterpret_cast<const float4*>(src1 + off);
      }
    }
#pragma unroll
    for (int k = 0; k < C; ++k) {
      const uint32_t q = q0 + threadIdx.x + k * kTileThreads;
      if (q < nq) {
        const uint32_t l = 2 * q;
        sm0[swz(l)] = make_float2(v0[k].x, v0[k].y);
        sm0[swz(l + 1)] = make_float2(v0[k].z, v0[k].w);
        if (TWO) {
          sm1[swz(l)] = make_float2(v1[k].x, v1[k].y);
          sm1[swz(l + 1)] = make_float2(v1[k].z, v1[k].w);
        }
      }
    }
  }
}

template <bool TWO>
__device__ __noinline__ void store_tiles(const float2* sm0, float2* dst0, const float2* sm1, float2* dst1,
                                         const uint32_t* rowoff, int m) {
  const uint32_t nq = 1u << (m - 1);
  for (uint32_t q = threadIdx.x; q < nq; q += kTileThreads) {
    const uint32_t off = rowoff[q >> 4] + 2 * (q & 15);
    const uint32_t l = 2 * q;
    const float2 a = sm0[swz(l)], b = sm0[swz(l + 1)];
    *reinterpret_cast<float4*>(dst0 + off) = make_float4(a.x, a.y, b.x, b.y);
    if (TWO) {
      const float2 c = sm1[swz(l)], d = sm1[swz(l + 1)];
      *reinterpret_cast<float4*>(dst1 + off) = make_float4(c.x, c.y, d.x, d.y);
    }
  }
}

__device__ __forceinline__ void load_tile(float2* sm, const float2* src, const uint32_t* rowoff, int m) {
  load_tiles<false>(sm, src, nullptr, nullptr, rowoff, m);
}
__device__ __forceinline__ void store_tile(const float2* sm, float2* dst, const uint32_t* rowoff, int m) {
  store_tiles<false>(sm, dst, nullptr, nullptr, rowoff, m);
}

// double-float tiles of psi and lambda (one float4 = hi.re, hi.im, lo.re, lo.im
// per amplitude, in global and shared memory)
__device__ __noinline__ void load_tiles_ff(float4* sm0, const float4* src0, float4* sm1, const float4* src1,
                                           const uint32_t* rowoff, int m) {
  const uint32_t cnt = 1u << m;
  constexpr int C = kLdChunk / 2;
  for (uint32_t q0 = 0; q0 < cnt; q0 += C * kTileThreads) {
    float4 v0[C], v1[C];
#pragma unroll
    for (int k = 0; k < C; ++k) {
      const uint32_t q = q0 + threadIdx.x + k * kTileThreads;
      if (q < cnt) {
        const uint32_t off = rowoff[q >> kRowBits] + (q & 31u);
        v0[k] = src0[off];
        v1[k] = src1[off];
      }
    }
#pragma unroll
    for (int k = 0; k < C; ++k) {
      const uint32_t q = q0 + threadIdx.x + k * kTileThreads;
      if (q < cnt) {
        sm0[swz(q)] = v0[k];
        sm1[swz(q)] = v1[k];
      }
    }
  }
}

__device__ __noinline__ void store_tiles_ff(const float4* sm0, float4* dst0, const float4* sm1, float4* dst1,
                                            const uint32_t* rowoff, int m) {
  const uint32_t cnt = 1u << m;
  for (uint32_t q = threadIdx.x; q < cnt; q += kTileThreads) {
    const uint32_t off = rowoff[q >> kRowBits] + (q & 31u);
    dst0[off] = sm0[swz(q)];
    dst1[off] = sm1[swz(q)];
  }
}

__device__ __forceinline__ uint32_t phase_base(uint32_t tid, const TPhase& ph, int nthreadbits) {
  uint32_t b = 0;
  for (int k = 0; k < nthreadbits; ++k) b |= ((tid >> k) & 1u) << ph.tpos[k];
  return b;
}

// global register index bits of this thread's amplitudes outside the phase
__device__ __forceinline__ uint32_t thread_global(uint32_t tid, const TPhase& ph, int nthreadbits, uint32_t tbase) {
  uint32_t b = tbase;
  for (int k = 0; k < nthreadbits; ++k) b |= ((tid >> k) & 1u) << ph.tq[k];
  return b;
}

// shared-memory slot of amplitude j of a phase: swz is linear over XOR, so
// slot(j) = swz(base) ^ (XOR of swz(offset of bit b) over the set bits b of j);
// the per-bit values stay in registers instead of reloading sroff[j]
struct PhaseSlots {
  uint32_t b, s0, s1, s2, s3;
};
__device__ __forceinline__ PhaseSlots phase_slots(uint32_t sb, const TPhase& ph) {
  return PhaseSlots{sb, ph.sroff[1], ph.sroff[2], ph.sroff[4], ph.sroff[8]};
}
__device__ __forceinline__ uint32_t slot(const PhaseSlots& p, int j) {
  uint32_t o = p.b;
  if (j & 1) o ^= p.s0;
  if (j & 2) o ^= p.s1;
  if (j & 4) o ^= p.s2;
  if (j & 8) o ^= p.s3;
  return o;
}

// An op record in registers from four 16-byte loads issued together: one
// memory latency per op, instead of a chain of dependent field loads behind
// the op's control test and kind branches
__device__ __forceinline__ TOp load_op(const TOp* p) {
  const uint4* s = reinterpret_cast<const uint4*>(p);
  const uint4 a = s[0], b = s[1], c = s[2], d = s[3];
  TOp r;
  r.kind = (uint8_t)(a.x & 0xffu);
  r.t = (uint8_t)((a.x >> 8) & 0xffu);
  r.cmask = (uint8_t)((a.x >> 16) & 0xffu);
  r.cval = (uint8_t)(a.x >> 24);
  r.gen = (uint8_t)(a.y & 0xffu);
  r.shared = (uint8_t)((a.y >> 8) & 0xffu);
  r.var = (uint8_t)((a.y >> 16) & 0xffu);
  r.pad = 0;
  r.param = (int32_t)a.z;
  r.cfac2 = __uint_as_float(a.w);
  r.tmask = b.x;
  r.tval = b.y;
  r.count = b.z;
  r.u[0] = make_float2(__uint_as_float(c.x), __uint_as_float(c.y));
  r.u[1] = make_float2(__uint_as_float(c.z), __uint_as_float(c.w));
  r.u[2] = make_float2(__uint_as_float(d.x), __uint_as_float(d.y));
  r.u[3] = make_float2(__uint_as_float(d.z), __uint_as_float(d.w));
  return r;
}

// ---- shared-memory copies of a pass's phase records and ops
//
// Every tile of a pass runs the same phases, so a CTA that streams tiles reads
// each op record once per tile.  Read from global memory, those records are
// evicted from L1 by the tile traffic and every op then waits on L2 before
// its first arithmetic (the records are read by a chain of dependent loads:
// the control test, the kind, the target, the matrix).  The pass's records are
// therefore copied into shared memory once per pass, with the phases' op
// indices rebased to the pass's first op.  A pass larger than the staging
// area keeps reading global memory.
constexpr int kStagePhases = 32;
constexpr int kStageOps = 512;
constexpr int kStageRuns = 256;
static_assert(sizeof(TOp) == 64 && sizeof(TOp) % 16 == 0, "TOp is copied as 16-byte words");
static_assert(sizeof(DRun) == 32, "DRun is copied as 16-byte words");
constexpr size_t kStagePhaseBytes = (sizeof(TPhase) * kStagePhases + 15) & ~size_t(15);
constexpr size_t kStageBytes = kStagePhaseBytes + sizeof(TOp) * kStageOps + sizeof(DRun) * kStageRuns;

struct StagedPass {
  const TPhase* ph;  // the pass's first phase
  const TOp* ops;    // op table the phases index
  int first;         // index of ops[0] in the global op table (0 when not staged)
  const DRun* runs;  // the pass's TK_DIAGRUN entries (forward)
};

// FWD: the forward ops (fop0 / nfop), else the backward ops (bop0 / nbop).
// buf: kStageBytes of shared memory, or nullptr.  Every thread of the CTA
// calls this (it ends with a barrier when it copies).
template <bool FWD>
__device__ StagedPass stage_pass(const TPass& p, const TPhase* phases, const TOp* ops, unsigned char* buf,
                                 const DRun* druns = nullptr) {
  StagedPass r{phases + p.phase0, ops, 0, druns ? druns + p.drun0 : nullptr};
  if (!buf || p.nphase <= 0 || p.nphase > kStagePhases) return r;
  if (FWD && druns && p.ndrun > kStageRuns) return r;
  const TPhase& f0 = phases[p.phase0];
  const TPhase& fl = phases[p.phase0 + p.nphase - 1];
  const int first = FWD ? f0.fop0 : f0.bop0;
  const int count = FWD ? fl.fop0 + fl.nfop - first : fl.bop0 + fl.nbop - first;
  if (count < 0 || count > kStageOps) return r;
  TPhase* sph = reinterpret_cast<TPhase*>(buf);
  TOp* sop = reinterpret_cast<TOp*>(buf + kStagePhaseBytes);
  constexpr int W = (int)(sizeof(TOp) / 16);
  const uint4* src = reinterpret_cast<const uint4*>(ops + first);
  uint4* dst = reinterpret_cast<uint4*>(sop);
  for (int i = threadIdx.x; i < count * W; i += blockDim.x) dst[i] = src[i];
  if ((int)threadIdx.x < p.nphase) {
    TPhase q = phases[p.phase0 + threadIdx.x];
    if (FWD) q.fop0 -= first;
    else q.bop0 -= first;
    sph[threadIdx.x] = q;
  }
  const DRun* runs = nullptr;
  if (FWD && druns) {
    DRun* srun = reinterpret_cast<DRun*>(buf + kStagePhaseBytes + sizeof(TOp) * kStageOps);
    const uint4* rs = reinterpret_cast<const uint4*>(druns + p.drun0);
    uint4* rd = reinterpret_cast<uint4*>(srun);
    for (int i = threadIdx.x; i < p.ndrun * 2; i += blockDim.x) rd[i] = rs[i];
    runs = srun;
  }
  __syncthreads();
  return StagedPass{sph, sop, first, runs};
}

// out-of-phase diagonal gate with phase-local controls: x_j *= f where (j & cm) == cv
template <int RB>
__device__ __forceinline__ void diag_masked(float2 (&x)[1 << RB], float2 f, int cm, int cv) {
#pragma unroll
  for (int j = 0; j < (1 << RB); ++j)
    if ((j & cm) == cv) x[j] = cmulf(x[j], f);
}

// COMP: compensated matrices (flo: 4 corrections per forward op, dtlo: 16 per
// diagonal table); out-of-phase diagonal factors are then applied one by one
template <int RB, bool COMP, bool RESLOT>
__device__ __forceinline__ void phase_fwd_body(float2* sm, const TPhase* php, const TOp* fops, const float2* dtab,
                                               const float2* flo, const float2* dtlo, const DRun* runs, int m,
                                               uint32_t tbase) {
  constexpr int A = 1 << RB;
  const TPhase& ph = *php;
  const int ntb = m - RB;
  if (threadIdx.x < (1u << ntb)) {
    const PhaseSlots ps = phase_slots(swz(phase_base(threadIdx.x, ph, ntb)), ph);
    const uint32_t gb = thread_global(threadIdx.x, ph, ntb, tbase);
    float2 x[A];
#pragma unroll
    for (int j = 0; j < A; ++j) x[j] = sm[slot(ps, j)];
    // factors of out-of-phase diagonal gates without phase-local controls are
    // scalars for this thread: they commute with the phase and are applied once
    float2 pend = make_float2(1.f, 0.f);
    bool has_pend = false;
    for (int o = 0; o < ph.nfop; ++o) {
      const int oi = ph.fop0 + o;
      const TOp cur = load_op(fops + oi);
      if ((gb & cur.tmask) != cur.tval) continue;
      if (cur.kind == TK_DIAGOUT) {
        const bool b1 = (gb >> cur.t) & 1u;
        const float2 f = b1 ? cur.u[3] : cur.u[0];
        if (COMP) {
          const float2 fl = flo[4 * oi + (b1 ? 3 : 0)];
#pragma unroll
          for (int j = 0; j < A; ++j)
            if ((j & cur.cmask) == cur.cval) x[j] = cf_mul(x[j], f, fl);
        } else if (f.x == 1.f && f.y == 0.f) {
          // a factor of exactly 1 (the |0> entry of a shift or controlled phase)
        } else if (cur.cmask == 0) {
          pend = cmulf(pend, f);
          has_pend = true;
        } else {
          diag_masked<RB>(x, f, cur.cmask, cur.cval);
        }
      } else if (cur.kind == TK_DIAG16) {
        const float2* t = dtab + 16 * cur.param;
        if (COMP) {
          const float2* tl = dtlo + 16 * cur.param;
#pragma unroll
          for (int j = 0; j < A; ++j) x[j] = cf_mul(x[j], t[j], tl[j]);
        } else {
#pragma unroll
          for (int j = 0; j < A; ++j) x[j] = cmulf(x[j], t[j]);
        }
      } else {
        apply_fwd_var<RB, COMP>(x, cur, COMP ? flo + 4 * oi : nullptr, runs, gb);
      }
    }
    if (!COMP && has_pend) {
#pragma unroll
      for (int j = 0; j < A; ++j) x[j] = cmulf(x[j], pend);
    }
    // RESLOT: the slot offsets again (from shared memory) rather than live
    // through the op loop (fewer spills in k_batch; slower in the tile engine,
    // whose loop does not spill)
    const PhaseSlots ps2 = RESLOT ? phase_slots(swz(phase_base(threadIdx.x, ph, ntb)), ph) : ps;
#pragma unroll
    for (int j = 0; j < A; ++j) sm[slot(ps2, j)] = x[j];
  }
  __syncthreads();
}

// All phases of a pass on one tile, in order (one call per tile).  SITE gives
// each call site its own copy: ptxas allocates a called function's registers
// per kernel, and one copy shared by the resident and streamed loops of
// k_batch spilled several times as much (ptxas -v) as two copies do; SITE 2
// is the tile engine's pass.
template <int RB, bool COMP, int SITE = 0>
__device__ __noinline__ void run_tile_fwd(float2* sm, const TPhase* ph, int nphase, const TOp* fops,
                                          const float2* dtab, const float2* flo, const float2* dtlo,
                                          const DRun* runs, int m, uint32_t tbase) {
  for (int f = 0; f < nphase; ++f)
    phase_fwd_body<RB, COMP, SITE != 2>(sm, ph + f, fops, dtab, flo, dtlo, runs, m, tbase);
}

// backward of an out-of-phase diagonal gate: the generator is diagonal on the
// target (Z, P1 or 1), whose value is fixed for this thread
__device__ __forceinline__ float diagout_sign(const TOp& op, bool b) {
  switch (op.gen) {
    case GEN_Z: return b ? -1.f : 1.f;
    case GEN_P1: return b ? 1.f : 0.f;
    case GEN_I: return 1.f;
    default: return 0.f;
  }
}

template <int RB>
__device__ __forceinline__ float diagout_bwd(float2 (&x)[1 << RB], float2 (&l)[1 << RB], const TOp& op, uint32_t gb) {
  const bool b = (gb >> op.t) & 1u;
  const float2 d = b ? op.u[3] : op.u[0];
  const int cm = op.cmask, cv = op.cval;
  float acc = 0.f;
#pragma unroll
  for (int j = 0; j < (1 << RB); ++j) {
    if ((j & cm) != cv) continue;
    acc += imcj(l[j], x[j]);
    x[j] = cmulf(x[j], d);
    l[j] = cmulf(l[j], d);
  }
  return diagout_sign(op, b) * acc;
}

template <int RB>
__device__ __forceinline__ float diagout_bwd_ff(ffc (&x)[1 << RB], ffc (&l)[1 << RB], const TOp& op, const float2* lo,
                                                uint32_t gb) {
  const bool b = (gb >> op.t) & 1u;
  const float2 d = b ? op.u[3] : op.u[0];
  const float2 dl = b ? lo[3] : lo[0];
  const int cm = op.cmask, cv = op.cval;
  float acc = 0.f;
#pragma unroll
  for (int j = 0; j < (1 << RB); ++j) {
    if ((j & cm) != cv) continue;
    acc += imcj(l[j].h, x[j].h);
    x[j] = ff_cmul(x[j], d, dl);
    l[j] = ff_cmul(l[j], d, dl);
  }
  return diagout_sign(op, b) * acc;
}

// Warp sums of the gradient ops' lane partials, two ops at a time: the two
// shuffle trees interleave, so a warp waits on one chain of shuffle latencies
// per pair of ops instead of per op.  pend / pend_o hold the first op of a pair
// (pend_o is the same in every lane).
__device__ __forceinline__ void warp_partial(float part, int o, float& pend, int& pend_o, float* red, int lane,
                                             int warp) {
  if (pend_o < 0) {
    pend = part;
    pend_o = o;
    return;
  }
#pragma unroll
  for (int s = 16; s > 0; s >>= 1) {
    pend += __shfl_xor_sync(0xffffffffu, pend, s);
    part += __shfl_xor_sync(0xffffffffu, part, s);
  }
  if (lane == 0) {
    red[pend_o * kWarps + warp] = pend;
    red[o * kWarps + warp] = part;
  }
  pend_o = -1;
}
__device__ __forceinline__ void flush_partial(float pend, int pend_o, float* red, int lane, int warp) {
  if (pend_o < 0) return;
#pragma unroll
  for (int s = 16; s > 0; s >>= 1) pend += __shfl_xor_sync(0xffffffffu, pend, s);
  if (lane == 0) red[pend_o * kWarps + warp] = pend;
}

// fold the warp partials of every parameterised op of a phase: the 16 warp
// partials of an op are summed by 16 lanes in a TwoSum tree (the double-float
// sum s + e of the FP32 partials, exact to ~2^-48), one op per 16 lanes, all
// ops at once; the leader adds (s + e) cfac2 to the FP64 accumulator.  Ops whose
// parameter another op of the phase shares are added by one thread afterwards.
// (FP64 arithmetic runs at 1/64 of the FP32 rate here: summing in FP64 took
// one warp thousands of cycles per phase while the others waited.)
__device__ __forceinline__ void fold_phase_grad(const TPhase& ph, const TOp* bops, const float* red, double* gacc) {
  static_assert(kWarps == 16, "one op per 16 lanes");
  const int nbop = ph.nbop, bop0 = ph.bop0;
  for (int base = 0; base < nbop * kWarps; base += blockDim.x) {
    const int t = base + (int)threadIdx.x;
    const int o = t >> 4, w = t & 15;
    const bool valid = o < nbop && bops[bop0 + o].gen != GEN_NONE;
    float s = valid ? red[o * kWarps + w] : 0.f, e = 0.f;
#pragma unroll
    for (int d = 8; d > 0; d >>= 1) {
      const float so = __shfl_xor_sync(0xffffffffu, s, d), eo = __shfl_xor_sync(0xffffffffu, e, d);
      float q, r;
      two_sum(s, so, q, r);
      s = q;
      e = __fadd_rn(__fadd_rn(e, eo), r);
    }
    if (w == 0 && valid) {
      const TOp& op = bops[bop0 + o];
      if (!op.shared) gacc[op.param] += (double)op.cfac2 * ((double)s + (double)e);
    }
  }
  __syncthreads();
  if (ph.nshared == 0) return;
  if (threadIdx.x == 0) {
    for (int q = 0; q < nbop; ++q) {
      const TOp& op = bops[bop0 + q];
      if (op.gen == GEN_NONE || !op.shared) continue;
      double v = 0.0;
      for (int w = 0; w < kWarps; ++w) v += (double)red[q * kWarps + w];
      gacc[op.param] += (double)op.cfac2 * v;
    }
  }
  __syncthreads();
}

template <int RB>
__device__ __forceinline__ void phase_bwd_body(float2* sx, float2* sl, const TPhase* php, const TOp* bops, int m,
                                               float* red, double* gacc, uint32_t tbase) {
  // the phase record is read where it lies (the pass's shared-memory copy when
  // staged): with 2 x 2^RB live amplitudes per thread there are no registers
  // to spare for a copy of it
  constexpr int A = 1 << RB;
  const TPhase& ph = *php;
  const int ntb = m - RB;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const bool active = threadIdx.x < (1u << ntb);
  const int nbop = ph.nbop, bop0 = ph.bop0;
  float2 x[A], l[A];
  const uint32_t gb = active ? thread_global(threadIdx.x, ph, ntb, tbase) : 0u;
  const PhaseSlots ps = phase_slots(active ? swz(phase_base(threadIdx.x, ph, ntb)) : 0u, ph);
  if (active) {
#pragma unroll
    for (int j = 0; j < A; ++j) {
      const uint32_t o = slot(ps, j);
      x[j] = sx[o];
      l[j] = sl[o];
    }
  }
  float pend = 0.f;  // warp partial of a gradient op waiting for a partner (pend_o >= 0)
  int pend_o = -1;
  for (int o = nbop - 1; o >= 0; --o) {
    const TOp op = load_op(bops + bop0 + o);
    float part = 0.f;
    if (active && (gb & op.tmask) == op.tval)
      part = op.kind == TK_DIAGOUT ? diagout_bwd<RB>(x, l, op, gb) : apply_bwd_var<RB>(x, l, op);
    if (op.gen != GEN_NONE) warp_partial(part, o, pend, pend_o, red, lane, warp);
  }
  flush_partial(pend, pend_o, red, lane, warp);
  if (active) {
#pragma unroll
    for (int j = 0; j < A; ++j) {
      const uint32_t o = slot(ps, j);
      sx[o] = x[j];
      sl[o] = l[j];
    }
  }
  __syncthreads();
  fold_phase_grad(ph, bops, red, gacc);
}

// All phases of a pass on one tile, last phase first: one call per tile, so
// that the callers' loop state is saved once per tile rather than per phase
template <int RB>
__device__ __noinline__ void run_tile_bwd(float2* sx, float2* sl, const TPhase* ph, int nphase, const TOp* bops,
                                          int m, float* red, double* gacc, uint32_t tbase) {
  for (int f = nphase - 1; f >= 0; --f) phase_bwd_body<RB>(sx, sl, ph + f, bops, m, red, gacc, tbase);
}

template <int RB>
__device__ __noinline__ void run_phase_bwd_ff(float4* sx, float4* sl, const TPhase* php, const TOp* bops,
                                              const float2* blo, int m, float* red, double* gacc, uint32_t tbase) {
  constexpr int A = 1 << RB;
  const TPhase& ph = *php;
  const int ntb = m - RB;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const bool active = threadIdx.x < (1u << ntb);
  const int nbop = ph.nbop, bop0 = ph.bop0;
  ffc x[A], l[A];
  const uint32_t gb = active ? thread_global(threadIdx.x, ph, ntb, tbase) : 0u;
  const PhaseSlots ps = phase_slots(active ? swz(phase_base(threadIdx.x, ph, ntb)) : 0u, ph);
  if (active) {
#pragma unroll
    for (int j = 0; j < A; ++j) {
      const uint32_t o = slot(ps, j);
      const float4 a = sx[o], b = sl[o];
      x[j].h = make_float2(a.x, a.y);
      x[j].l = make_float2(a.z, a.w);
      l[j].h = make_float2(b.x, b.y);
      l[j].l = make_float2(b.z, b.w);
    }
  }
  float pend = 0.f;
  int pend_o = -1;
  for (int o = nbop - 1; o >= 0; --o) {
    const int oi = bop0 + o;
    const TOp op = load_op(bops + oi);
    float part = 0.f;
    if (active && (gb & op.tmask) == op.tval)
      part = op.kind == TK_DIAGOUT ? diagout_bwd_ff<RB>(x, l, op, blo + 4 * oi, gb)
                                   : apply_bwd_ff<RB>(x, l, op, blo + 4 * oi);
    if (op.gen != GEN_NONE) warp_partial(part, o, pend, pend_o, red, lane, warp);
  }
  flush_partial(pend, pend_o, red, lane, warp);
  if (active) {
#pragma unroll
    for (int j = 0; j < A; ++j) {
      const uint32_t o = slot(ps, j);
      sx[o] = make_float4(x[j].h.x, x[j].h.y, x[j].l.x, x[j].l.y);
      sl[o] = make_float4(l[j].h.x, l[j].h.y, l[j].l.x, l[j].l.y);
    }
  }
  __syncthreads();
  fold_phase_grad(ph, bops, red, gacc);
}

// the diagonal observable's weight w(i) = sum_t c_t (-1)^popcount(i & z_t)
__device__ __forceinline__ double obs_weight(uint64_t gi, const BTerm* terms, int nterm) {
  double w = 0.0;
  for (int t = 0; t < nterm; ++t) w += (__popcll(gi & terms[t].z) & 1) ? -terms[t].coeff : terms[t].coeff;
  return w;
}

// loss partial and lambda = w psi for the diagonal observable, over a tile in smem
__device__ double expect_tile(float2* sx, float2* sl, uint64_t tbase, const uint32_t* rowoff, int m,
                              const BTerm* terms, int nterm) {
  const uint32_t cnt = 1u << m;
  double acc = 0.0;
  for (uint32_t l = threadIdx.x; l < cnt; l += blockDim.x) {
    const uint64_t gi = tbase + rowoff[l >> kRowBits] + (l & 31u);
    const double w = obs_weight(gi, terms, nterm);
    const float2 a = sx[swz(l)];
    acc += w * ((double)a.x * a.x + (double)a.y * a.y);
    const float wf = (float)w;
    sl[swz(l)] = make_float2(wf * a.x, wf * a.y);
  }
  return acc;
}

// the same from a complex64 tile into double-float psi and lambda tiles
// (w psi formed in FP64 and split into hi + lo)
__device__ double expect_tile_ff(const float2* s2, float4* sxf, float4* slf, uint64_t tbase, const uint32_t* rowoff,
                                 int m, const BTerm* terms, int nterm) {
  const uint32_t cnt = 1u << m;
  double acc = 0.0;
  for (uint32_t l = threadIdx.x; l < cnt; l += blockDim.x) {
    const uint64_t gi = tbase + rowoff[l >> kRowBits] + (l & 31u);
    const double w = obs_weight(gi, terms, nterm);
    const float2 a = s2[swz(l)];
    acc += w * ((double)a.x * a.x + (double)a.y * a.y);
    const double lr = w * (double)a.x, li = w * (double)a.y;
    const float hr = (float)lr, hi = (float)li;
    sxf[swz(l)] = make_float4(a.x, a.y, 0.f, 0.f);
    slf[swz(l)] = make_float4(hr, hi, (float)(lr - (double)hr), (float)(li - (double)hi));
  }
  return acc;
}

__device__ void block_loss(double e, BShared& S, double* out) {
  for (int s = 16; s > 0; s >>= 1) e += __shfl_xor_sync(0xffffffffu, e, s);
  if ((threadIdx.x & 31) == 0) S.lred[threadIdx.x >> 5] = e;
  __syncthreads();
  if (threadIdx.x == 0) {
    static_assert(kWarps == 16, "loss tree below is written for 16 warps");
    const double* v = S.lred;
    *out = (((v[0] + v[1]) + (v[2] + v[3])) + ((v[4] + v[5]) + (v[6] + v[7]))) +
           (((v[8] + v[9]) + (v[10] + v[11])) + ((v[12] + v[13]) + (v[14] + v[15])));
  }
}

// The per-register phase loops of k_batch live in their own (not inlined)
// functions: a phase call then sees only the loop's few live values, and the
// phase functions keep their amplitudes in registers.
template <int RB>
__device__ __noinline__ void batch_bwd_resident(float2* sx, float2* sl, const TPass* P, int npass, int m,
                                                const TPhase* phases, const TOp* bops, float* red, double* gacc) {
  for (int pi = npass - 1; pi >= 0; --pi)
    run_tile_bwd<RB>(sx, sl, phases + P[pi].phase0, P[pi].nphase, bops, m, red, gacc, 0u);
}

template <int RB>
__device__ __noinline__ void batch_bwd_resident_ff(float4* sx, float4* sl, const TPass* P, int npass, int m,
                                                   const TPhase* phases, const TOp* bops, const float2* blo,
                                                   float* red, double* gacc) {
  for (int pi = npass - 1; pi >= 0; --pi) {
    const int ph0 = P[pi].phase0;
    for (int f = P[pi].nphase - 1; f >= 0; --f)
      run_phase_bwd_ff<RB>(sx, sl, phases + ph0 + f, bops, blo, m, red, gacc, 0u);
  }
}

template <int RB>
__device__ __noinline__ void batch_bwd_streamed(float2* sx, float2* sl, const TPass* P, int npass, int m, int g,
                                                float2* wp, float2* wl, const TPhase* phases, const TOp* bops,
                                                uint32_t* rowoff, float* red, double* gacc, unsigned char* stage) {
  const uint64_t ntile = 1ull << g;
  for (int pi = npass - 1; pi >= 0; --pi) {
    const TPass& p = P[pi];
    set_rows(rowoff, p, m);
    const StagedPass sp = stage_pass<false>(p, phases, bops, stage);
    for (uint64_t t = 0; t < ntile; ++t) {
      const uint64_t tb = tile_base(t, p, g);
      load_tiles<true>(sx, wp + tb, sl, wl + tb, rowoff, m);
      __syncthreads();
      run_tile_bwd<RB>(sx, sl, sp.ph, p.nphase, sp.ops, m, red, gacc, (uint32_t)tb);
      store_tiles<true>(sx, wp + tb, sl, wl + tb, rowoff, m);
      __syncthreads();
    }
  }
}

template <int RB>
__device__ __noinline__ void batch_bwd_streamed_ff(float4* sx, float4* sl, const TPass* P, int npass, int m, int g,
                                                   float4* wp, float4* wl, const TPhase* phases, const TOp* bops,
                                                   const float2* blo, uint32_t* rowoff, float* red, double* gacc,
                                                   unsigned char* stage) {
  const uint64_t ntile = 1ull << g;
  for (int pi = npass - 1; pi >= 0; --pi) {
    const TPass& p = P[pi];
    set_rows(rowoff, p, m);
    const StagedPass sp = stage_pass<false>(p, phases, bops, stage);
    const float2* lo = blo + 4 * (size_t)sp.first;
    for (uint64_t t = 0; t < ntile; ++t) {
      const uint64_t tb = tile_base(t, p, g);
      load_tiles_ff(sx, wp + tb, sl, wl + tb, rowoff, m);
      __syncthreads();
      for (int f = p.nphase - 1; f >= 0; --f)
        run_phase_bwd_ff<RB>(sx, sl, sp.ph + f, sp.ops, lo, m, red, gacc, (uint32_t)tb);
      store_tiles_ff(sx, wp + tb, sl, wl + tb, rowoff, m);
      __syncthreads();
    }
  }
}

// cp.async copies (8 bytes each: the swizzled slots of a 16-byte pair may be
// swapped) of the next tile into a second buffer while the current one is computed
__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
  const uint32_t d = (uint32_t)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_prev() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// issue the copies of one tile (2^m amplitudes) into sm (no wait)
__device__ __forceinline__ void load_tile_async(float2* sm, const float2* src, const uint32_t* rowoff, int m) {
  const uint32_t n = 1u << m;
  for (uint32_t l = threadIdx.x; l < n; l += kTileThreads)
    cp_async8(sm + swz(l), src + rowoff[l >> kRowBits] + (l & 31u));
}

template <int RB, bool COMP>
__device__ __noinline__ void batch_fwd_streamed(float2* sx, float2* sx2, float2* st, const TPass* P, int npass,
                                                int m, int g, const TPhase* phases, const TOp* fops,
                                                const float2* dtab, const float2* flo, const float2* dtlo,
                                                const DRun* druns, uint32_t* rowoff, unsigned char* stage) {
  const uint64_t ntile = 1ull << g;
  for (int pi = 0; pi < npass; ++pi) {
    const TPass& p = P[pi];
    set_rows(rowoff, p, m);
    const StagedPass sp = stage_pass<true>(p, phases, fops, stage, druns);
    const float2* lo = COMP ? flo + 4 * (size_t)sp.first : nullptr;
    // two tile buffers (sx, sx2): the next tile's copies are in flight while
    // the current one is computed
    load_tile_async(sx, st + tile_base(0, p, g), rowoff, m);
    cp_async_commit();
    for (uint64_t t = 0; t < ntile; ++t) {
      float2* cur = (t & 1) ? sx2 : sx;
      if (t + 1 < ntile) load_tile_async((t & 1) ? sx : sx2, st + tile_base(t + 1, p, g), rowoff, m);
      cp_async_commit();
      cp_async_wait_prev();
      __syncthreads();
      const uint64_t tb = tile_base(t, p, g);
      run_tile_fwd<RB, COMP, 1>(cur, sp.ph, p.nphase, sp.ops, dtab, lo, dtlo, sp.runs, m, (uint32_t)tb);
      store_tile(cur, st + tb, rowoff, m);
      __syncthreads();
    }
    cp_async_wait_all();
  }
}

// CTAs per SM the register budget is sized for (two CTAs of 3-qubit phases, at
// 64 registers a thread, spilled and measured slower: 247 vs 213 ms per batch)
template <int RB, bool PREC>
constexpr int kBatchMinBlocks = 1;

// Shared memory of k_batch after the BShared header: the complex64 path holds
// psi and lambda tiles (2 x 2^13 x 8 bytes); the precise path holds double-float
// psi and lambda tiles (2 x 2^m x 16 bytes) and a complex64 forward tile.
template <int RB, bool PREC>
__global__ void __launch_bounds__(kTileThreads, kBatchMinBlocks<RB, PREC>) k_batch(BArgs a) {
  extern __shared__ __align__(16) unsigned char smraw[];
  BShared& S = *reinterpret_cast<BShared*>(smraw);
  constexpr int MT = kTileThreads == 512 ? 9 + RB : 0;  // largest tile: 512 threads x 2^RB amplitudes
  static_assert(MT >= kRowBits + RB && MT <= kMaxTileBits, "tile size");
  unsigned char* body = smraw + ((sizeof(BShared) + 255) & ~size_t(255));
  float2* sx = reinterpret_cast<float2*>(body);                   // complex64 psi tile (forward, and FP32 backward)
  float2* sl = sx + (1 << MT);                                    // complex64 lambda tile (FP32 backward)
  float4* sxf = reinterpret_cast<float4*>(body + (size_t)8 * (1 << MT));   // double-float psi (precise)
  float4* slf = sxf + (1 << MT);                                           // double-float lambda (precise)
  unsigned char* stage = body + (size_t)(PREC ? 40 : 16) * (1 << MT);      // a pass's records (streamed registers)
  const int tid = threadIdx.x;
  for (;;) {
    if (tid == 0) S.reg = atomicAdd(a.counter, 1);
    __syncthreads();
    const int ri = S.reg;
    __syncthreads();
    if (ri >= a.nreg) break;
    const int reg = a.order[ri];
    const BReg R = a.regs[reg];
    const int n = R.n, m = R.m, g = n - m;
    const bool grad = (a.flags & BF_GRAD) != 0;
    for (int i = tid; i < R.nparam; i += blockDim.x) S.grad[i] = 0.0;
    float2* st = a.state + R.amp_off;
    const uint64_t ntile = 1ull << g;
    const TPass* P = a.passes + R.pass0;
    if (g == 0) {
      // ---- whole register in shared memory
      set_rows(S.rowoff, P[0], m);
      if (a.flags & BF_RESET) {
        for (uint32_t l = tid; l < (1u << m); l += blockDim.x) sx[swz(l)] = make_float2(l == 0 ? 1.f : 0.f, 0.f);
      } else {
        load_tile(sx, st, S.rowoff, m);
      }
      __syncthreads();
      for (int pi = 0; pi < R.npass; ++pi)
        run_tile_fwd<RB, PREC>(sx, a.phases + P[pi].phase0, P[pi].nphase, a.fops, a.dtab, a.flo, a.dtlo,
                               a.druns + P[pi].drun0, m, 0u);
      store_tile(sx, st, S.rowoff, m);  // psi_N
      if (PREC) {
        block_loss(expect_tile_ff(sx, sxf, slf, 0, S.rowoff, m, a.terms + R.term0, R.nterm), S, a.loss + reg);
        __syncthreads();
        if (grad) batch_bwd_resident_ff<RB>(sxf, slf, P, R.npass, m, a.phases, a.bops, a.blo, S.red, S.grad);
      } else {
        block_loss(expect_tile(sx, sl, 0, S.rowoff, m, a.terms + R.term0, R.nterm), S, a.loss + reg);
        __syncthreads();
        if (grad) batch_bwd_resident<RB>(sx, sl, P, R.npass, m, a.phases, a.bops, S.red, S.grad);
      }
    } else {
      // ---- tiles streamed through global memory
      if (a.flags & BF_RESET) {
        for (uint64_t i = tid; i < (1ull << n); i += blockDim.x) st[i] = make_float2(i == 0 ? 1.f : 0.f, 0.f);
        __syncthreads();
      }
      batch_fwd_streamed<RB, PREC>(sx, PREC ? reinterpret_cast<float2*>(sxf) : sl, st, P, R.npass, m, g, a.phases,
                                   a.fops, a.dtab, a.flo, a.dtlo, a.druns, S.rowoff, stage);
      // expectation, lambda = O psi, and the work copy of psi for the uncompute
      double e = 0.0;
      const TPass& p0 = P[0];
      set_rows(S.rowoff, p0, m);
      for (uint64_t t = 0; t < ntile; ++t) {
        const uint64_t tb = tile_base(t, p0, g);
        load_tile(sx, st + tb, S.rowoff, m);
        __syncthreads();
        if (PREC) {
          e += expect_tile_ff(sx, sxf, slf, tb, S.rowoff, m, a.terms + R.term0, R.nterm);
          __syncthreads();
          if (grad) store_tiles_ff(sxf, a.wpsif + R.work_off + tb, slf, a.wlamf + R.work_off + tb, S.rowoff, m);
        } else {
          e += expect_tile(sx, sl, tb, S.rowoff, m, a.terms + R.term0, R.nterm);
          __syncthreads();
          if (grad) store_tiles<true>(sx, a.wpsi + R.work_off + tb, sl, a.wlam + R.work_off + tb, S.rowoff, m);
        }
        __syncthreads();
      }
      block_loss(e, S, a.loss + reg);
      __syncthreads();
      if (grad) {
        if (PREC)
          batch_bwd_streamed_ff<RB>(sxf, slf, P, R.npass, m, g, a.wpsif + R.work_off, a.wlamf + R.work_off, a.phases,
                                    a.bops, a.blo, S.rowoff, S.red, S.grad, stage);
        else
          batch_bwd_streamed<RB>(sx, sl, P, R.npass, m, g, a.wpsi + R.work_off, a.wlam + R.work_off, a.phases,
                                 a.bops, S.rowoff, S.red, S.grad, stage);
      }
    }
    __syncthreads();
    if (grad)
      for (int i = tid; i < R.nparam; i += blockDim.x) a.grad[R.param_off + i] = S.grad[i];
    __syncthreads();
  }
}

// bytes of dynamic shared memory of k_batch<RB, PREC>
static size_t batch_smem(int rb, bool prec) {
  const size_t mt = (size_t)1 << (9 + rb);
  return ((sizeof(BShared) + 255) & ~size_t(255)) + (prec ? (8 + 32) * mt : 16 * mt) + kStageBytes;
}

// the instantiation of k_batch for a phase width and path
static const void* batch_kernel(int rb, bool prec) {
  if (prec) return rb == 2 ? (const void*)k_batch<2, true> : (const void*)k_batch<3, true>;
  switch (rb) {
    case 2: return (const void*)k_batch<2, false>;
    case 3: return (const void*)k_batch<3, false>;
    default: return (const void*)k_batch<4, false>;
  }
}


// ------------------------------------------------------------------ device: fused forward passes of large registers

struct FArgs {
  float2* state;
  const TPass* pass;
  const TPhase* phases;
  const TOp* fops;
  const float2* dtab;
  const DRun* druns;
  int m, g;
  uint64_t ntile;          // tiles per register
  uint64_t reg_stride;     // amplitudes per register
  int nreg;
};

// One pass over every register of a uniform batch: CTA-strided over tiles,
// each tile staged in shared memory once and run through all phases of the pass.
//
// Two tile buffers: the next tile's amplitudes are copied into one with
// cp.async (8-byte copies into the swizzled slots) while the phases run on the
// other, so the pass does not wait on the state's DRAM latency once per tile.
__global__ void __launch_bounds__(kTileThreads, 1) k_fused_pass(FArgs a) {
  extern __shared__ __align__(16) unsigned char smraw[];
  uint32_t* rowoff = reinterpret_cast<uint32_t*>(smraw);
  float2* sbuf = reinterpret_cast<float2*>(smraw + sizeof(uint32_t) * (1 << (kMaxTileBits - kRowBits)));
  unsigned char* stage = reinterpret_cast<unsigned char*>(sbuf + 2 * (1 << kBatchTile));
  const TPass& p = *a.pass;
  set_rows(rowoff, p, a.m);
  const StagedPass sp = stage_pass<true>(p, a.phases, a.fops, stage, a.druns);
  const uint64_t total = a.ntile * (uint64_t)a.nreg;
  auto tile_src = [&](uint64_t t, uint64_t& tb) {
    const uint64_t r = t / a.ntile, tl = t - r * a.ntile;
    tb = tile_base(tl, p, a.g);
    return a.state + r * a.reg_stride + tb;
  };
  uint64_t tb = 0;
  if (blockIdx.x < total) load_tile_async(sbuf, tile_src(blockIdx.x, tb), rowoff, a.m);
  cp_async_commit();
  int i = 0;
  for (uint64_t t = blockIdx.x; t < total; t += gridDim.x, ++i) {
    float2* sx = sbuf + (size_t)(i & 1) * (1 << kBatchTile);
    const uint64_t tn = t + gridDim.x;
    if (tn < total) {
      uint64_t tbn;
      load_tile_async(sbuf + (size_t)((i + 1) & 1) * (1 << kBatchTile), tile_src(tn, tbn), rowoff, a.m);
    }
    cp_async_commit();
    cp_async_wait_prev();  // this tile's copies (all groups but the one just issued)
    __syncthreads();
    float2* base = tile_src(t, tb);
    run_tile_fwd<kRB, false, 2>(sx, sp.ph, p.nphase, sp.ops, a.dtab, nullptr, nullptr, sp.runs, a.m, (uint32_t)tb);
    store_tile(sx, base, rowoff, a.m);
    __syncthreads();
  }
  cp_async_wait_all();
}


// One backward pass over a single large register (complex64 psi and lambda
// work copies): CTA-strided over tiles; every CTA accumulates the pass's
// gradient contributions in its own FP64 shared-memory slots and writes them
// to partials[blockIdx.x][param]; k_fold_partials sums the CTAs in order.
struct FBArgs {
  float2* wpsi;
  float2* wlam;
  const TPass* pass;
  const TPhase* phases;
  const TOp* bops;
  int m, g, nparam;
  int stage;             // 1: kStageBytes of shared memory after the tiles hold the pass's records
  uint64_t ntile;
  double* partials;      // [gridDim.x][nparam]
};

__global__ void __launch_bounds__(kTileThreads, 1) k_fused_bwd_pass(FBArgs a) {
  extern __shared__ __align__(16) unsigned char smraw[];
  uint32_t* rowoff = reinterpret_cast<uint32_t*>(smraw);
  float* red = reinterpret_cast<float*>(rowoff + (1 << (kMaxTileBits - kRowBits)));
  double* gacc = reinterpret_cast<double*>(red + kMaxPhaseOps * kWarps);
  float2* sx = reinterpret_cast<float2*>(gacc + ((a.nparam + 1) & ~1));
  float2* sl = sx + (1 << a.m);
  unsigned char* stage = a.stage ? reinterpret_cast<unsigned char*>(sl + (1 << a.m)) : nullptr;
  const TPass& p = *a.pass;
  for (int i = threadIdx.x; i < a.nparam; i += blockDim.x) gacc[i] = 0.0;
  set_rows(rowoff, p, a.m);
  const StagedPass sp = stage_pass<false>(p, a.phases, a.bops, stage);
  for (uint64_t t = blockIdx.x; t < a.ntile; t += gridDim.x) {
    const uint64_t tb = tile_base(t, p, a.g);
    load_tiles<true>(sx, a.wpsi + tb, sl, a.wlam + tb, rowoff, a.m);
    __syncthreads();
    run_tile_bwd<kRB>(sx, sl, sp.ph, p.nphase, sp.ops, a.m, red, gacc, (uint32_t)tb);
    store_tiles<true>(sx, a.wpsi + tb, sl, a.wlam + tb, rowoff, a.m);
    __syncthreads();
  }
  for (int i = threadIdx.x; i < a.nparam; i += blockDim.x) a.partials[(size_t)blockIdx.x * a.nparam + i] = gacc[i];
}

__global__ void k_fold_partials(const double* __restrict__ partials, int nblk, int nparam, double* __restrict__ grad) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nparam) return;
  double v = 0.0;
  for (int b = 0; b < nblk; ++b) v += partials[(size_t)b * nparam + i];
  grad[i] += v;
}

// lambda = O psi for complex64 work copies (FP32 arithmetic, FP64 coefficients)
struct ObsC64 {
  int nt;
  uint64_t x[64];
  uint64_t z[64];
  int ny[64];
  float c[64];
};

__global__ void __launch_bounds__(256) k_apply_obs_c64(const float2* __restrict__ psi, float2* __restrict__ lam,
                                                       uint64_t dim, int accumulate, const __grid_constant__ ObsC64 o) {
  const uint64_t i = (uint64_t)blockIdx.x * 256 + threadIdx.x;
  if (i >= dim) return;
  float2 acc = accumulate ? lam[i] : make_float2(0.f, 0.f);
  for (int t = 0; t < o.nt; ++t) {
    const uint64_t j = i ^ o.x[t];
    const float2 v = psi[j];
    const float s = (__popcll(j & o.z[t]) & 1) ? -o.c[t] : o.c[t];
    float re, im;
    switch (o.ny[t] & 3) {
      case 0: re = v.x; im = v.y; break;
      case 1: re = -v.y; im = v.x; break;
      case 2: re = -v.x; im = -v.y; break;
      default: re = v.y; im = -v.x; break;
    }
    acc.x = fmaf(s, re, acc.x);
    acc.y = fmaf(s, im, acc.y);
  }
  lam[i] = acc;
}

// ------------------------------------------------------------------ device: matrices from parameters

// member of a TK_DIAG16 table: a diagonal gate on the phase bits
struct DMem {
  int32_t g;                 // global GSpec index
  uint8_t tb, cm, cv, pad;   // phase-local target bit, control mask and values
};

struct DRef {
  int32_t mem0, count;       // members in dmem[]
};

struct PrepArgs {
  const GSpec* gspec;
  const FMem* fmem;
  const int32_t* bgate;
  float2* flo;             // if not NULL: corrections of the forward matrices (precise path)
  float2* blo;             // backward U^dagger corrections
  float2* dtlo;            // diagonal table corrections
  const DMem* dmem;
  const DRef* dref;
  TOp* fops;
  TOp* bops;
  float2* dtab;
  DRun* druns;
  const double* params;
  int nfop, nbop, ndiag, ndrun;
};

__device__ void gate_mat(const GSpec& gs, const double* params, double2 (&U)[4]) {
  const double th = gs.param >= 0 ? params[gs.param] : gs.theta;
  double s, c;
  sincos(th * 0.5, &s, &c);
  const double h = 0.70710678118654752440;
  auto set = [&](double a0, double a1, double b0, double b1, double c0, double c1, double d0, double d1) {
    U[0] = make_double2(a0, a1); U[1] = make_double2(b0, b1); U[2] = make_double2(c0, c1); U[3] = make_double2(d0, d1);
  };
  switch (gs.kind) {
    case QS_GATE_X: set(0, 0, 1, 0, 1, 0, 0, 0); break;
    case QS_GATE_Y: set(0, 0, 0, -1, 0, 1, 0, 0); break;
    case QS_GATE_Z: set(1, 0, 0, 0, 0, 0, -1, 0); break;
    case QS_GATE_H: set(h, 0, h, 0, h, 0, -h, 0); break;
    case QS_GATE_S: set(1, 0, 0, 0, 0, 0, 0, 1); break;
    case QS_GATE_SDG: set(1, 0, 0, 0, 0, 0, 0, -1); break;
    case QS_GATE_T: set(1, 0, 0, 0, 0, 0, h, h); break;
    case QS_GATE_TDG: set(1, 0, 0, 0, 0, 0, h, -h); break;
    case QS_GATE_RX: set(c, 0, 0, -s, 0, -s, c, 0); break;
    case QS_GATE_RY: set(c, 0, -s, 0, s, 0, c, 0); break;
    case QS_GATE_RZ: set(c, -s, 0, 0, 0, 0, c, s); break;
    case QS_GATE_SHIFT: { double s2, c2; sincos(th, &s2, &c2); set(1, 0, 0, 0, 0, 0, c2, s2); break; }
    case QS_GATE_PHASE: { double s2, c2; sincos(th, &s2, &c2); set(c2, s2, 0, 0, 0, 0, c2, s2); break; }
    case QS_GATE_MATRIX: U[0] = gs.mat[0]; U[1] = gs.mat[1]; U[2] = gs.mat[2]; U[3] = gs.mat[3]; break;
    default: set(1, 0, 0, 0, 0, 0, 1, 0); break;
  }
}

__device__ __forceinline__ double2 zmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 zadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }

// FP32 value of v and its correction v - hi (both components)
__device__ __forceinline__ float2 hi_of(double2 v) { return make_float2((float)v.x, (float)v.y); }
__device__ __forceinline__ float2 lo_of(double2 v) {
  const float2 h = hi_of(v);
  return make_float2((float)(v.x - (double)h.x), (float)(v.y - (double)h.y));
}

__global__ void k_batch_prep(PrepArgs a) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < a.nfop) {
    const FMem& fm = a.fmem[i];
    double2 A[4] = {make_double2(1, 0), make_double2(0, 0), make_double2(0, 0), make_double2(1, 0)};
    for (int k = 0; k < fm.count; ++k) {
      double2 U[4];
      gate_mat(a.gspec[fm.g[k]], a.params, U);
      const double2 C0 = zadd(zmul(U[0], A[0]), zmul(U[1], A[2]));
      const double2 C1 = zadd(zmul(U[0], A[1]), zmul(U[1], A[3]));
      const double2 C2 = zadd(zmul(U[2], A[0]), zmul(U[3], A[2]));
      const double2 C3 = zadd(zmul(U[2], A[1]), zmul(U[3], A[3]));
      A[0] = C0; A[1] = C1; A[2] = C2; A[3] = C3;
    }
    for (int k = 0; k < 4; ++k) a.fops[i].u[k] = hi_of(A[k]);
    if (a.flo)
      for (int k = 0; k < 4; ++k) a.flo[4 * i + k] = lo_of(A[k]);
  } else if (i < a.nfop + a.nbop) {
    const int j = i - a.nfop;
    double2 U[4];
    gate_mat(a.gspec[a.bgate[j]], a.params, U);
    // U^dagger
    const double2 D[4] = {make_double2(U[0].x, -U[0].y), make_double2(U[2].x, -U[2].y),
                          make_double2(U[1].x, -U[1].y), make_double2(U[3].x, -U[3].y)};
    for (int k = 0; k < 4; ++k) a.bops[j].u[k] = hi_of(D[k]);
    if (a.blo)
      for (int k = 0; k < 4; ++k) a.blo[4 * j + k] = lo_of(D[k]);
  } else if (i < a.nfop + a.nbop + a.ndiag) {
    // product of the member gates' diagonals on the 16 phase amplitudes
    const int d = i - a.nfop - a.nbop;
    double2 f[16];
    for (int j = 0; j < 16; ++j) f[j] = make_double2(1.0, 0.0);
    const DRef r = a.dref[d];
    for (int k = 0; k < r.count; ++k) {
      const DMem mb = a.dmem[r.mem0 + k];
      double2 U[4];
      gate_mat(a.gspec[mb.g], a.params, U);
      for (int j = 0; j < 16; ++j)
        if ((j & mb.cm) == mb.cv) f[j] = zmul(f[j], ((j >> mb.tb) & 1) ? U[3] : U[0]);
    }
    for (int j = 0; j < 16; ++j) a.dtab[16 * d + j] = hi_of(f[j]);
    if (a.dtlo)
      for (int j = 0; j < 16; ++j) a.dtlo[16 * d + j] = lo_of(f[j]);
  } else if (i < a.nfop + a.nbop + a.ndiag + a.ndrun) {
    DRun& e = a.druns[i - a.nfop - a.nbop - a.ndiag];
    double2 U[4];
    gate_mat(a.gspec[e.gate], a.params, U);
    e.u0 = hi_of(U[0]);
    e.u3 = hi_of(U[3]);
  }
}

}  // namespace qs

// ------------------------------------------------------------------ host: the program object

struct qs_batch_program {
  int device = -1;                   // CUDA device that holds the tables below
  int nreg = 0;
  std::vector<int> nq;
  std::vector<int64_t> param_off;    // nreg + 1
  std::vector<int64_t> amp_off;      // nreg + 1
  int64_t work_elems = 0;
  // device tables
  qs::BReg* regs = nullptr;
  int32_t* order = nullptr;
  qs::TPass* passes = nullptr;
  qs::TPhase* phases = nullptr;
  qs::TOp* fops = nullptr;
  qs::TOp* bops = nullptr;
  qs::BTerm* terms = nullptr;
  qs::GSpec* gspec = nullptr;
  qs::FMem* fmem = nullptr;
  int32_t* bgate = nullptr;
  qs::DMem* dmem = nullptr;
  qs::DRef* dref = nullptr;
  float2* dtab = nullptr;
  int ndiag = 0;
  qs::DRun* druns = nullptr;  // TK_DIAGRUN entries
  int ndrun = 0;
  int* counter = nullptr;
  float2* wpsi = nullptr;
  float2* wlam = nullptr;
  // phase width and the precise path (compensated forward, double-float uncompute)
  int rb = qs::kRB;
  int tile = 0;
  bool precise = false;
  float2* flo = nullptr;   // corrections of the forward ops (4 per op)
  float2* blo = nullptr;   // corrections of the backward ops (4 per op)
  float2* dtlo = nullptr;  // corrections of the diagonal tables (16 per table)
  float4* wpsif = nullptr;
  float4* wlamf = nullptr;
  int nfop = 0, nbop = 0;
  int64_t npass = 0, nphase = 0;
  int blocks = 0;
  size_t smem = 0;
  // single-register fused forward (no observable, no backward): host copies of
  // the pass table and a device parameter buffer
  bool fused_only = false;
  std::vector<qs::TPass> host_passes;
  double* dparams = nullptr;
  int64_t dparams_n = 0;
};

namespace qs {

static bool diag_kind(int k) {
  return k == QS_GATE_Z || k == QS_GATE_S || k == QS_GATE_SDG || k == QS_GATE_T || k == QS_GATE_TDG ||
         k == QS_GATE_RZ || k == QS_GATE_SHIFT || k == QS_GATE_PHASE || k == QS_GATE_I;
}

static int gen_of(int kind, float* cfac2) {
  switch (kind) {
    case QS_GATE_RX: *cfac2 = 1.f; return GEN_X;
    case QS_GATE_RY: *cfac2 = 1.f; return GEN_Y;
    case QS_GATE_RZ: *cfac2 = 1.f; return GEN_Z;
    case QS_GATE_SHIFT: *cfac2 = -2.f; return GEN_P1;
    case QS_GATE_PHASE: *cfac2 = -2.f; return GEN_I;
  }
  *cfac2 = 0.f;
  return GEN_NONE;
}

template <typename T>
static int upload(T** dst, const std::vector<T>& v) {
  const size_t bytes = sizeof(T) * std::max<size_t>(1, v.size());
  if (cudaMalloc((void**)dst, bytes) != cudaSuccess) {
    cudaGetLastError();
    *dst = nullptr;
    return fail(QS_ENOMEM, "cudaMalloc of %zu program bytes failed", bytes);
  }
  if (!v.empty()) QS_CUDA(cudaMemcpy(*dst, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice));
  return QS_OK;
}

static void free_program(qs_batch_program* p) {
  if (!p) return;
  // the tables live on the device that built them, which need not be the current one
  int cur = -1;
  const bool swap = p->device >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != p->device &&
                    cudaSetDevice(p->device) == cudaSuccess;
  void* ptrs[] = {p->regs, p->order, p->passes, p->phases, p->fops, p->bops, p->terms, p->gspec, p->fmem,
                  p->bgate, p->dmem, p->dref, p->dtab, p->counter, p->wpsi, p->wlam, p->dparams,
                  p->flo, p->blo, p->dtlo, p->wpsif, p->wlamf, p->druns};
  for (void* q : ptrs)
    if (q) cudaFree(q);
  if (swap) cudaSetDevice(cur);
  delete p;
}

// largest tile of the batched kernel for rb-bit phases: 512 threads x 2^rb amplitudes
static int max_tile(int rb) { return std::min(kBatchTile, 9 + rb); }

// TOp::var of a backward op (bwd_form): 13 t + form
static uint8_t bwd_variant(const TOp& b) {
  if (b.kind == TK_DIAGOUT) return 0xff;
  int f;
  if (b.gen == GEN_NONE) f = b.kind == TK_SWAP ? 0 : b.kind == TK_DIAG ? 1 : 2;
  else f = 3 + 2 * (b.gen - GEN_X) + (b.cmask ? 1 : 0);
  return (uint8_t)(13 * b.t + f);
}

// TOp::var of a forward op (FV_* forms)
static uint8_t fwd_variant(const TOp& f) {
  switch (f.kind) {
    case TK_DIAGOUT: return FV_DIAGOUT;
    case TK_DIAG16: return FV_DIAG16;
    case TK_DIAGRUN: return FV_DIAGRUN;
    case TK_SWAP: return (uint8_t)(FV_SWAP + f.t);
    case TK_DIAG: return (uint8_t)((f.cmask ? FV_DIAGC : FV_DIAG) + f.t);
    default: return (uint8_t)((f.cmask ? FV_DENSEC : FV_DENSE) + f.t);
  }
}

static int build_program(int nreg, const qs_circuit* const* circs, const qs_observable* const* obs, int tile_qubits,
                         qs_batch_program* P, int rb = kRB, bool precise = false) {
  if (rb < kMinRB || rb > kRB) return fail(QS_EINVAL, "phase_qubits must be in %d..%d", kMinRB, kRB);
  if (precise && rb > 3) return fail(QS_EINVAL, "the precise path takes phases of at most 3 qubits");
  const int MT = max_tile(rb);
  const int M = tile_qubits > 0 ? tile_qubits : MT;
  // a tile holds register qubits 0..4 (contiguous rows) plus a phase's register bits
  if (M < kRowBits + rb || M > MT)
    return fail(QS_EINVAL, "tile_qubits must be in %d..%d for %d-qubit phases", kRowBits + rb, MT, rb);
  P->rb = rb;
  P->precise = precise;
  P->tile = M;
  QS_CUDA(cudaGetDevice(&P->device));
  std::vector<BReg> regs(nreg);
  std::vector<TPass> passes;
  std::vector<TPhase> phases;
  std::vector<TOp> fops, bops;
  std::vector<BTerm> terms;
  std::vector<GSpec> gspec;
  std::vector<FMem> fmem;
  std::vector<int32_t> bgate;
  std::vector<DMem> dmems;
  std::vector<DRef> drefs;
  std::vector<DRun> druns;
  P->nreg = nreg;
  P->nq.resize(nreg);
  P->param_off.assign(nreg + 1, 0);
  P->amp_off.assign(nreg + 1, 0);
  int64_t work = 0;
  for (int r = 0; r < nreg; ++r) {
    const qs_circuit* c = circs[r];
    const qs_observable* o = obs ? obs[r] : nullptr;
    if (!c || (!o && !P->fused_only)) return fail(QS_EINVAL, "register %d: null circuit or observable", r);
    const int n = c->nqubits;
    if (n < kRowBits || n > (P->fused_only ? 32 : 30))
      return fail(QS_EUNSUPPORTED, "register %d: %d qubits outside the tile engine's range", r, n);
    if (!P->fused_only && c->nparams > kMaxRegParams)
      return fail(QS_EUNSUPPORTED, "register %d: more than %d parameters", r, kMaxRegParams);
    P->nq[r] = n;
    P->param_off[r + 1] = P->param_off[r] + c->nparams;
    P->amp_off[r + 1] = P->amp_off[r] + (1ll << n);
    const int m = std::min(n, M);
    std::vector<HostPass> hp;
    QS_TRY(plan_passes(c, n, m, kMaxPhaseOps, hp, rb));
    BReg& R = regs[r];
    memset(&R, 0, sizeof(R));
    R.n = n;
    R.m = m;
    R.npass = (int)hp.size();
    R.pass0 = (int)passes.size();
    R.nparam = c->nparams;
    R.amp_off = P->amp_off[r];
    R.param_off = P->param_off[r];
    R.work_off = (n > m && !P->fused_only) ? work : -1;
    if (n > m && !P->fused_only) work += 1ll << n;
    // observable: diagonal Pauli strings only
    R.term0 = (int)terms.size();
    if (o) {
      for (const auto& t : o->terms) {
        if (t.x_mask) return fail(QS_EUNSUPPORTED, "register %d: batched observables must be diagonal (Z strings)", r);
        if (n < 64 && (t.z_mask >> n)) return fail(QS_EINVAL, "register %d: observable qubit out of range", r);
        terms.push_back({t.coeff, t.z_mask});
      }
    }
    R.nterm = o ? (int)o->terms.size() : 0;
    // gate specs of this register
    const int g0 = (int)gspec.size();
    for (const auto& g : c->gates) {
      GSpec s;
      memset(&s, 0, sizeof(s));
      s.kind = g.kind;
      s.param = g.param >= 0 ? (int)(P->param_off[r] + g.param) : -1;
      s.theta = g.theta;
      if (g.kind == QS_GATE_MATRIX) {
        if (g.nlocs != 1) return fail(QS_EUNSUPPORTED, "register %d: multi-qubit matrices in a batch", r);
        for (int k = 0; k < 4; ++k) s.mat[k] = make_double2(c->mats[g.mat_offset + k].real(), c->mats[g.mat_offset + k].imag());
      }
      if (g.kind == QS_GATE_ROT || g.kind == QS_GATE_SWAP)
        return fail(QS_EUNSUPPORTED, "register %d: ROT / SWAP gates in a batch", r);
      gspec.push_back(s);
    }
    double cost = 0;
    for (const HostPass& p : hp) {
      TPass tp;
      memset(&tp, 0, sizeof(tp));
      for (int k = 0; k < m; ++k) tp.tbits[k] = (uint8_t)p.tbits[k];
      int ng = 0;
      for (int qb = 0; qb < n; ++qb)
        if (std::find(p.tbits.begin(), p.tbits.end(), qb) == p.tbits.end()) tp.gbits[ng++] = (uint8_t)qb;
      tp.phase0 = (int)phases.size();
      tp.drun0 = (int)druns.size();
      tp.nphase = (int)p.phases.size();
      for (const HostPhase& ph : p.phases) {
        TPhase t;
        phase_positions(p, ph, &t, rb);
        // register qubit -> phase bit index
        auto pbit = [&](int qb) {
          for (int k = 0; k < rb; ++k)
            if (ph.rbits[k] == qb) return k;
          return -1;
        };
        t.bop0 = (int)bops.size();
        t.fop0 = (int)fops.size();
        std::vector<int> last(rb, -1);   // forward op index (in fops) open for fusion per phase bit
        int dg = -1;                     // open TK_DIAG16 table of this phase
        // TK_DIAGRUN runs of this phase (complex64 path): the op each opened,
        // its entries, the run open per phase bit and the latest run opened
        std::vector<int> run_op;
        std::vector<std::vector<DRun>> run_ent;
        std::vector<int> run_bit;
        std::vector<int> run_open(rb, -1);
        int run_last = -1;
        uint8_t nondiag = 0;             // phase bits touched by non-diagonal gates since it opened
        for (int gi : ph.gates) {
          const qs_gate_desc& g = c->gates[gi];
          const bool diag = gate_is_diagonal(c, g);
          const int tb = pbit(g.locs[0]);  // -1: target outside the phase (diagonal gates only)
          uint8_t cm = 0, cv = 0;          // controls inside the phase
          uint32_t tmask = 0, tval = 0;    // controls outside the phase (register qubits)
          for (int qb = 0; qb < n; ++qb)
            if ((g.ctrl_mask >> qb) & 1ull) {
              const int k = pbit(qb);
              const bool v = (g.ctrl_vals >> qb) & 1ull;
              if (k >= 0) {
                cm |= (uint8_t)(1 << k);
                if (v) cv |= (uint8_t)(1 << k);
              } else {
                tmask |= 1u << qb;
                if (v) tval |= 1u << qb;
              }
            }
          // backward op: one per gate
          TOp b;
          memset(&b, 0, sizeof(b));
          b.t = (uint8_t)(tb >= 0 ? tb : g.locs[0]);
          b.cmask = cm;
          b.cval = cv;
          b.tmask = tmask;
          b.tval = tval;
          b.param = g.param;
          b.gen = g.param >= 0 ? (uint8_t)gen_of(g.kind, &b.cfac2) : GEN_NONE;
          // uncompute kind: the generator picks the structured form (Rx / Ry / diagonal)
          if (tb < 0) b.kind = TK_DIAGOUT;
          else if (b.gen == GEN_X) b.kind = TK_RX;
          else if (b.gen == GEN_Y) b.kind = TK_RY;
          else if (b.gen != GEN_NONE) b.kind = TK_DIAG;
          else b.kind = g.kind == QS_GATE_X ? TK_SWAP : diag ? TK_DIAG : TK_DENSE;
          if (g.param >= 0 && b.gen == GEN_NONE)
            return fail(QS_EUNSUPPORTED, "register %d gate %d: kind %d has no batched gradient", r, gi, g.kind);
          for (int q = t.bop0; q < (int)bops.size(); ++q)
            if (bops[q].gen != GEN_NONE && b.gen != GEN_NONE && bops[q].param == b.param) {
              bops[q].shared = 1;
              b.shared = 1;
            }
          bops.push_back(b);
          bgate.push_back(g0 + gi);
          // forward op.  A diagonal gate with its target outside the phase is a
          // per-thread factor.  Consecutive uncontrolled gates on one target fuse
          // into one 2x2; controlled diagonal gates inside the phase join its open
          // 16-entry table unless a non-diagonal op since the table opened shares a
          // qubit with them (diagonal gates commute with each other).
          TOp f;
          memset(&f, 0, sizeof(f));
          f.cmask = cm;
          f.cval = cv;
          f.tmask = tmask;
          f.tval = tval;
          f.param = -1;
          FMem fm;
          memset(&fm, 0, sizeof(fm));
          fm.count = 1;
          fm.g[0] = g0 + gi;
          if (tb < 0 && !precise && cm == 0 && run_last >= 0 && run_open[run_bit[run_last]] == run_last) {
            // a scalar for each thread: commutes with every op of the phase
            DRun e;
            memset(&e, 0, sizeof(e));
            e.tmask = tmask;
            e.tval = tval;
            e.gate = g0 + gi;
            e.tq = (uint32_t)g.locs[0];
            run_ent[run_last].push_back(e);
            continue;
          }
          if (tb < 0) {
            f.kind = TK_DIAGOUT;
            f.t = (uint8_t)g.locs[0];
            fops.push_back(f);
            fmem.push_back(fm);
            for (int k = 0; k < rb; ++k)
              if ((cm >> k) & 1) last[k] = -1;
            continue;
          }
          const bool fusable = cm == 0 && tmask == 0 && g.kind != QS_GATE_X;
          const uint8_t gbits = (uint8_t)(cm | (1u << tb));
          if (!diag) nondiag |= gbits;
          if (!diag) run_open[tb] = -1;  // a run moves no later gate past this one
          if (fusable && last[tb] >= 0 && fmem[last[tb]].count < 4) {
            FMem& fmo = fmem[last[tb]];
            fmo.g[fmo.count++] = g0 + gi;
            if (!diag) fops[last[tb]].kind = TK_DENSE;
          } else if (!precise && diag && cm == 0 && tmask != 0) {
            // joins (or opens) the run on its target: diagonal gates commute, and
            // no non-diagonal op on this bit was emitted since the run opened
            if (run_open[tb] < 0) {
              f.kind = TK_DIAGRUN;
              f.t = (uint8_t)tb;
              f.tmask = f.tval = 0;
              fm.count = 0;
              run_open[tb] = (int)run_op.size();
              run_last = run_open[tb];
              run_op.push_back((int)fops.size());
              run_ent.emplace_back();
              run_bit.push_back(tb);
              fops.push_back(f);
              fmem.push_back(fm);
            }
            DRun e;
            memset(&e, 0, sizeof(e));
            e.tmask = tmask;
            e.tval = tval;
            e.gate = g0 + gi;
            e.tq = 0xffffffffu;
            run_ent[run_open[tb]].push_back(e);
          } else if (diag && cm != 0 && tmask == 0) {
            if (dg < 0 || (gbits & nondiag)) {
              f.kind = TK_DIAG16;
              f.cmask = f.cval = 0;
              f.param = (int)drefs.size();
              fm.count = 0;
              fops.push_back(f);
              fmem.push_back(fm);
              drefs.push_back({(int32_t)dmems.size(), 0});
              dg = (int)drefs.size() - 1;
              nondiag = 0;
            }
            DMem mb;
            memset(&mb, 0, sizeof(mb));
            mb.g = g0 + gi;
            mb.tb = (uint8_t)tb;
            mb.cm = cm;
            mb.cv = cv;
            dmems.push_back(mb);
            drefs[dg].count++;
          } else {
            f.kind = g.kind == QS_GATE_X ? TK_SWAP : diag ? TK_DIAG : TK_DENSE;
            f.t = (uint8_t)tb;
            fops.push_back(f);
            fmem.push_back(fm);
            last[tb] = fusable ? (int)fops.size() - 1 : -1;
          }
          // a controlled gate closes fusion on its target and its phase-local controls
          if (cm || tmask) {
            for (int k = 0; k < rb; ++k)
              if ((cm >> k) & 1) last[k] = -1;
            last[tb] = -1;
          }
        }
        for (size_t r = 0; r < run_op.size(); ++r) {
          TOp& ro = fops[run_op[r]];
          if (run_ent[r].size() == 1) {
            // a run of one gate stays that gate's own op (its outside controls as tmask)
            const DRun& e = run_ent[r][0];
            ro.kind = TK_DIAG;
            ro.tmask = e.tmask;
            ro.tval = e.tval;
            ro.param = -1;
            fmem[run_op[r]].count = 1;
            fmem[run_op[r]].g[0] = e.gate;
            continue;
          }
          ro.param = (int)druns.size() - tp.drun0;
          ro.count = (uint32_t)run_ent[r].size();
          druns.insert(druns.end(), run_ent[r].begin(), run_ent[r].end());
        }
        t.nbop = (int)bops.size() - t.bop0;
        t.nfop = (int)fops.size() - t.fop0;
        t.nshared = 0;
        for (int q = t.bop0; q < (int)bops.size(); ++q) t.nshared += bops[q].shared ? 1 : 0;
        if (t.nbop > kMaxPhaseOps) return fail(QS_EUNSUPPORTED, "phase with %d ops", t.nbop);
        phases.push_back(t);
        cost += (double)(1ll << n) * (1 + 0.02 * t.nbop);
      }
      tp.ndrun = (int)druns.size() - tp.drun0;
      passes.push_back(tp);
    }
    R.cost = cost;
  }
  for (TOp& f : fops) f.var = fwd_variant(f);
  for (TOp& b : bops) b.var = bwd_variant(b);
  // decreasing cost order
  std::vector<int32_t> order(nreg);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return regs[a].cost > regs[b].cost; });
  P->nfop = (int)fops.size();
  P->nbop = (int)bops.size();
  P->npass = (int64_t)passes.size();
  P->nphase = (int64_t)phases.size();
  P->work_elems = work;
  QS_TRY(upload(&P->regs, regs));
  QS_TRY(upload(&P->order, order));
  QS_TRY(upload(&P->passes, passes));
  QS_TRY(upload(&P->phases, phases));
  QS_TRY(upload(&P->fops, fops));
  QS_TRY(upload(&P->bops, bops));
  QS_TRY(upload(&P->terms, terms));
  QS_TRY(upload(&P->gspec, gspec));
  QS_TRY(upload(&P->fmem, fmem));
  QS_TRY(upload(&P->bgate, bgate));
  QS_TRY(upload(&P->dmem, dmems));
  QS_TRY(upload(&P->dref, drefs));
  P->ndiag = (int)drefs.size();
  P->ndrun = (int)druns.size();
  QS_TRY(upload(&P->druns, druns.empty() ? std::vector<DRun>(1) : druns));
  QS_TRY(upload(&P->dtab, std::vector<float2>(16 * std::max<size_t>(1, drefs.size()))));
  QS_TRY(upload(&P->counter, std::vector<int>(1, 0)));
  if (work > 0 && !precise) {
    if (cudaMalloc(&P->wpsi, sizeof(float2) * work) != cudaSuccess ||
        cudaMalloc(&P->wlam, sizeof(float2) * work) != cudaSuccess) {
      cudaGetLastError();
      return fail(QS_ENOMEM, "cudaMalloc of the backward work buffers failed");
    }
  }
  if (precise) {
    if ((work > 0 && (cudaMalloc(&P->wpsif, sizeof(float4) * work) != cudaSuccess ||
                      cudaMalloc(&P->wlamf, sizeof(float4) * work) != cudaSuccess)) ||
        cudaMalloc(&P->flo, sizeof(float2) * 4 * std::max<size_t>(1, fops.size())) != cudaSuccess ||
        cudaMalloc(&P->blo, sizeof(float2) * 4 * std::max<size_t>(1, bops.size())) != cudaSuccess ||
        cudaMalloc(&P->dtlo, sizeof(float2) * 16 * std::max<size_t>(1, drefs.size())) != cudaSuccess) {
      cudaGetLastError();
      return fail(QS_ENOMEM, "cudaMalloc of the precise path's buffers failed");
    }
  }
  P->host_passes = passes;
  if (P->fused_only) {
    P->smem = sizeof(uint32_t) * (1 << (kMaxTileBits - kRowBits)) + 2 * sizeof(float2) * (1 << kBatchTile) + kStageBytes;
    QS_CUDA(cudaFuncSetAttribute(k_fused_pass, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)P->smem));
    int dev = 0, sms = 0, per_sm = 0;
    QS_CUDA(cudaGetDevice(&dev));
    QS_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    QS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fused_pass, kTileThreads, P->smem));
    if (per_sm < 1) return fail(QS_EDEVICE, "fused pass kernel does not fit on an SM");
    P->blocks = sms * per_sm;
    return QS_OK;
  }
  P->smem = batch_smem(rb, precise);
  const void* kfn = batch_kernel(rb, precise);
  QS_CUDA(cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)P->smem));
  int dev = 0, sms = 0, per_sm = 0;
  QS_CUDA(cudaGetDevice(&dev));
  QS_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  QS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kfn, kTileThreads, P->smem));
  if (per_sm < 1) return fail(QS_EDEVICE, "batched kernel does not fit on an SM");
  P->blocks = std::min(nreg, sms * per_sm);
  return QS_OK;
}

// matrices of the forward ops, U^dagger of the backward ops (when `bwd`) and the
// diagonal tables from the current parameters, on the device
static int launch_prep(const qs_batch_program* P, const double* dev_params, bool bwd, cudaStream_t st) {
  PrepArgs pa;
  pa.gspec = P->gspec;
  pa.fmem = P->fmem;
  pa.bgate = P->bgate;
  pa.flo = P->flo;
  pa.blo = P->blo;
  pa.dtlo = P->dtlo;
  pa.dmem = P->dmem;
  pa.dref = P->dref;
  pa.fops = P->fops;
  pa.bops = P->bops;
  pa.dtab = P->dtab;
  pa.druns = P->druns;
  pa.params = dev_params;
  pa.nfop = P->nfop;
  pa.nbop = bwd ? P->nbop : 0;
  pa.ndiag = P->ndiag;
  pa.ndrun = P->ndrun;
  const int tot = pa.nfop + pa.nbop + pa.ndiag + pa.ndrun;
  if (tot > 0) {
    k_batch_prep<<<(tot + 255) / 256, 256, 0, st>>>(pa);
    QS_LAUNCHED();
  }
  return QS_OK;
}

// ------------------------------------------------------------------ host: fused forward of one circuit

// SWAP(a, b) = CX(a->b) CX(b->a) CX(a->b), each also carrying the SWAP's own controls
static void expand_swaps(const qs_circuit* c, qs_circuit* out) {
  out->nqubits = c->nqubits;
  out->nparams = c->nparams;
  out->mats = c->mats;
  out->gates.clear();
  for (const qs_gate_desc& g : c->gates) {
    if (g.kind != QS_GATE_SWAP) {
      out->gates.push_back(g);
      continue;
    }
    const int a = g.locs[0], b = g.locs[1];
    for (int k = 0; k < 3; ++k) {
      qs_gate_desc x;
      memset(&x, 0, sizeof(x));
      x.kind = QS_GATE_X;
      x.nlocs = 1;
      x.param = -1;
      const int t = (k == 1) ? a : b, ctl = (k == 1) ? b : a;
      x.locs[0] = t;
      x.ctrl_mask = g.ctrl_mask | (1ull << ctl);
      x.ctrl_vals = (g.ctrl_vals & g.ctrl_mask) | (1ull << ctl);
      out->gates.push_back(x);
    }
  }
}

// the circuit's tile-engine schedule for tiles of M qubits, built once and cached
// on the current device (a schedule built on another device is rebuilt here: its
// tables are that device's memory)
static int ensure_schedule(const qs_circuit* c, int M) {
  int dev = 0;
  QS_CUDA(cudaGetDevice(&dev));
  if (c->fused && c->fused_tile == M && c->fused->device == dev) return QS_OK;
  if (c->fused) {
    free_program(c->fused);
    c->fused = nullptr;
  }
  qs_circuit tmp;
  expand_swaps(c, &tmp);
  const qs_circuit* cp = &tmp;
  qs_batch_program* P = new qs_batch_program();
  P->fused_only = true;
  const int rc = build_program(1, &cp, nullptr, M, P);
  if (rc != QS_OK) {
    const std::string msg = qs_last_error();
    free_program(P);
    return fail(rc, "%s", msg.c_str());
  }
  c->fused = P;
  c->fused_tile = M;
  return QS_OK;
}

// Applies circuit c to the (uniform, complex64) registers of s with the tile
// engine: one launch of k_fused_pass per pass.  Returns QS_EUNSUPPORTED (with
// nothing launched) when the circuit does not fit the engine.
int fused_forward(qs_state* s, const qs_circuit* c, const double* host_params, int tile_qubits) {
  if (s->dtype != QS_C64 || !s->uniform || s->nq[0] != c->nqubits)
    return fail(QS_EUNSUPPORTED, "the tile engine runs uniform complex64 registers of the circuit's size");
  const int n = s->nq[0];
  const int M = tile_qubits > 0 ? tile_qubits : kBatchTile;
  QS_TRY(ensure_schedule(c, M));
  qs_batch_program* P = c->fused;
  cudaStream_t st = s->stream;
  if (c->nparams > 0) {
    if (P->dparams_n < c->nparams) {
      if (P->dparams) cudaFree(P->dparams);
      P->dparams = nullptr;
      P->dparams_n = 0;
      if (cudaMalloc(&P->dparams, sizeof(double) * c->nparams) != cudaSuccess) {
        cudaGetLastError();
        return fail(QS_ENOMEM, "cudaMalloc of the parameter buffer failed");
      }
      P->dparams_n = c->nparams;
    }
    QS_CUDA(cudaMemcpyAsync(P->dparams, host_params, sizeof(double) * c->nparams, cudaMemcpyHostToDevice, st));
  }
  QS_TRY(launch_prep(P, P->dparams, false, st));
  const int m = std::min(n, M), g = n - m;
  FArgs a;
  a.state = (float2*)s->data;
  a.phases = P->phases;
  a.fops = P->fops;
  a.dtab = P->dtab;
  a.druns = P->druns;
  a.m = m;
  a.g = g;
  a.ntile = 1ull << g;
  a.reg_stride = 1ull << n;
  a.nreg = s->nreg;
  const uint64_t tiles = a.ntile * (uint64_t)s->nreg;
  const unsigned grid = (unsigned)std::min<uint64_t>(tiles, (uint64_t)P->blocks);
  for (int64_t pi = 0; pi < P->npass; ++pi) {
    a.pass = P->passes + pi;
    k_fused_pass<<<grid, kTileThreads, P->smem, st>>>(a);
    QS_LAUNCHED();
  }
  return QS_OK;
}

void free_fused(qs_batch_program* p) { free_program(p); }

int schedule_info(const qs_circuit* c, int tile_qubits, int* npasses, int* nphases) {
  QS_TRY(ensure_schedule(c, tile_qubits > 0 ? tile_qubits : kBatchTile));
  if (npasses) *npasses = (int)c->fused->npass;
  if (nphases) *nphases = (int)c->fused->nphase;
  return QS_OK;
}

int tile_order(const qs_circuit* c, int tile_qubits, std::vector<int>& order, std::vector<int>& pass) {
  const int M = tile_qubits > 0 ? tile_qubits : kBatchTile;
  if (M < kRowBits + kRB || M > kBatchTile) return fail(QS_EINVAL, "tile_qubits must be in %d..%d", kRowBits + kRB, kBatchTile);
  const int n = c->nqubits;
  if (n < kRowBits || n > 32) return fail(QS_EUNSUPPORTED, "%d qubits outside the tile engine's range", n);
  qs_circuit tmp;
  expand_swaps(c, &tmp);
  std::vector<HostPass> hp;
  QS_TRY(plan_passes(&tmp, n, std::min(n, M), kMaxPhaseOps, hp));
  order.clear();
  pass.clear();
  for (size_t p = 0; p < hp.size(); ++p)
    for (const HostPhase& ph : hp[p].phases)
      for (int gi : ph.gates) {
        order.push_back(gi);
        pass.push_back((int)p);
      }
  return QS_OK;
}

int expect_raw(const void* data, int dtype, int n, int nreg, const qs_observable* o, qs_state* ws_owner,
               double* host_out);

// Reversible gradient of one complex64 register with the tile engine: psi_N and
// lambda = O psi_N are copied into dev_work (2 x 2^n complex64), then the
// schedule's passes run backwards (FP32 uncompute, FP64 accumulation of the
// per-CTA gradient partials, folded in CTA order).
int fused_backward(qs_state* s, const qs_circuit* c, const double* host_params, const qs_observable* o,
                   void* dev_work, double* host_grad, double* host_loss, int tile_qubits) {
  if (s->dtype != QS_C64 || s->nreg != 1 || s->nq[0] != c->nqubits)
    return fail(QS_EUNSUPPORTED, "the tiled backward takes one complex64 register of the circuit's size");
  if (!dev_work) return fail(QS_EINVAL, "work buffer is NULL");
  const int n = s->nq[0];
  const int M = tile_qubits > 0 ? tile_qubits : kBatchTile;
  const int m = std::min(n, M), g = n - m;
  for (const auto& t : o->terms)
    if (n < 64 && ((t.x_mask | t.z_mask) >> n)) return fail(QS_EINVAL, "observable acts on a qubit >= n=%d", n);
  if (o->terms.size() > 64) return fail(QS_EUNSUPPORTED, "the tiled backward takes at most 64 observable terms");
  // schedule (shared with the fused forward) and parameter-dependent matrices
  QS_TRY(ensure_schedule(c, M));
  qs_batch_program* P = c->fused;
  cudaStream_t st = s->stream;
  const int np = c->nparams;
  size_t smem = sizeof(uint32_t) * (1 << (kMaxTileBits - kRowBits)) + sizeof(float) * kMaxPhaseOps * kWarps +
                sizeof(double) * ((np + 1) & ~1) + 2 * sizeof(float2) * (1ull << m);
  if (smem > 227 * 1024) return fail(QS_EUNSUPPORTED, "%d parameters do not fit the tiled backward's shared memory", np);
  const bool stage = smem + kStageBytes <= 227 * 1024;
  if (stage) smem += kStageBytes;
  if (host_loss) QS_TRY(expect_raw(s->data, QS_C64, n, 1, o, s, host_loss));
  if (np > 0) {
    if (P->dparams_n < np) {
      if (P->dparams) cudaFree(P->dparams);
      P->dparams = nullptr;
      P->dparams_n = 0;
      if (cudaMalloc(&P->dparams, sizeof(double) * np) != cudaSuccess) {
        cudaGetLastError();
        return fail(QS_ENOMEM, "cudaMalloc of the parameter buffer failed");
      }
      P->dparams_n = np;
    }
    QS_CUDA(cudaMemcpyAsync(P->dparams, host_params, sizeof(double) * np, cudaMemcpyHostToDevice, st));
  }
  QS_TRY(launch_prep(P, P->dparams, true, st));
  // psi and lambda work copies
  const uint64_t dim = 1ull << n;
  float2* wpsi = (float2*)dev_work;
  float2* wlam = wpsi + dim;
  QS_CUDA(cudaMemcpyAsync(wpsi, s->data, sizeof(float2) * dim, cudaMemcpyDeviceToDevice, st));
  if (o->terms.empty()) {
    QS_CUDA(cudaMemsetAsync(wlam, 0, sizeof(float2) * dim, st));
  } else {
    ObsC64 ob;
    memset(&ob, 0, sizeof(ob));
    ob.nt = (int)o->terms.size();
    for (int t = 0; t < ob.nt; ++t) {
      ob.x[t] = o->terms[t].x_mask;
      ob.z[t] = o->terms[t].z_mask;
      ob.ny[t] = __builtin_popcountll(o->terms[t].x_mask & o->terms[t].z_mask) & 3;
      ob.c[t] = (float)o->terms[t].coeff;
    }
    k_apply_obs_c64<<<(unsigned)((dim + 255) / 256), 256, 0, st>>>(wpsi, wlam, dim, 0, ob);
    QS_LAUNCHED();
  }
  // per-CTA partials and the gradient accumulator in the state's scratch
  QS_CUDA(cudaFuncSetAttribute(k_fused_bwd_pass, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int dev = 0, sms = 0, per_sm = 0;
  QS_CUDA(cudaGetDevice(&dev));
  QS_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  QS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fused_bwd_pass, kTileThreads, smem));
  if (per_sm < 1) return fail(QS_EDEVICE, "tiled backward kernel does not fit on an SM");
  const uint64_t ntile = 1ull << g;
  const int grid = (int)std::min<uint64_t>(ntile, (uint64_t)sms * per_sm);
  const size_t npad = (size_t)std::max(1, np);
  QS_TRY(ensure_ws(s, s->ws, sizeof(double) * (npad + (size_t)grid * npad)));
  double* dgrad = (double*)s->ws.ptr;
  double* partials = dgrad + npad;
  QS_CUDA(cudaMemsetAsync(dgrad, 0, sizeof(double) * npad, st));
  FBArgs a;
  a.wpsi = wpsi;
  a.wlam = wlam;
  a.phases = P->phases;
  a.bops = P->bops;
  a.m = m;
  a.g = g;
  a.nparam = np;
  a.stage = stage ? 1 : 0;
  a.ntile = ntile;
  a.partials = partials;
  for (int64_t pi = P->npass - 1; pi >= 0; --pi) {
    a.pass = P->passes + pi;
    k_fused_bwd_pass<<<grid, kTileThreads, smem, st>>>(a);
    QS_LAUNCHED();
    if (np > 0) {
      k_fold_partials<<<(np + 255) / 256, 256, 0, st>>>(partials, grid, np, dgrad);
      QS_LAUNCHED();
    }
  }
  if (np > 0) QS_CUDA(cudaMemcpyAsync(host_grad, dgrad, sizeof(double) * np, cudaMemcpyDeviceToHost, st));
  QS_CUDA(cudaStreamSynchronize(st));
  return QS_OK;
}

}  // namespace qs

using namespace qs;

extern "C" {

int qs_batch_autotune(int nreg, const qs_circuit* const* circuits, const qs_observable* const* observables,
                      qs_state* s, const double* dev_params, double* dev_loss, double* dev_grad, int reps,
                      int* best_tile, int* ncand, int32_t* host_tiles, double* host_ms) {
  if (!circuits || !observables || !s || !dev_params || !dev_loss || !best_tile) return fail(QS_EINVAL, "null argument");
  if (reps < 1) reps = 1;
  const int flags = QS_BATCH_RESET | (dev_grad ? QS_BATCH_GRAD : 0);
  int best = -1, nc = 0;
  double best_ms = 0;
  cudaEvent_t e0, e1;
  QS_CUDA(cudaEventCreate(&e0));
  QS_CUDA(cudaEventCreate(&e1));
  int rc = QS_OK;
  for (int m = kBatchTile; m >= kRowBits + kRB + 2 && rc == QS_OK; --m) {
    qs_batch_program* P = nullptr;
    double ms = -1;
    const int crc = qs_batch_program_create(nreg, circuits, observables, m, &P);
    if (crc == QS_OK) {
      rc = qs_batch_run(s, P, dev_params, dev_loss, dev_grad, flags);  // warm-up
      if (rc == QS_OK && cudaEventRecord(e0, s->stream) != cudaSuccess) rc = fail(QS_EDEVICE, "event record");
      for (int r = 0; r < reps && rc == QS_OK; ++r) rc = qs_batch_run(s, P, dev_params, dev_loss, dev_grad, flags);
      if (rc == QS_OK && cudaEventRecord(e1, s->stream) != cudaSuccess) rc = fail(QS_EDEVICE, "event record");
      if (rc == QS_OK && cudaEventSynchronize(e1) != cudaSuccess) rc = fail(QS_EDEVICE, "event sync");
      float t = 0;
      if (rc == QS_OK && cudaEventElapsedTime(&t, e0, e1) == cudaSuccess) ms = (double)t / reps;
      qs_batch_program_destroy(P);
    } else if (crc != QS_EUNSUPPORTED && crc != QS_EINVAL) {
      rc = crc;
    }
    if (ncand && nc < *ncand) {
      if (host_tiles) host_tiles[nc] = m;
      if (host_ms) host_ms[nc] = ms;
    }
    ++nc;
    if (ms >= 0 && (best < 0 || ms < best_ms)) {
      best = m;
      best_ms = ms;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != QS_OK) return rc;
  if (ncand) *ncand = nc;
  if (best < 0) return fail(QS_EUNSUPPORTED, "no tile size ran the batch");
  *best_tile = best;
  return QS_OK;
}

int qs_batch_program_create(int nreg, const qs_circuit* const* circuits, const qs_observable* const* observables,
                            int tile_qubits, qs_batch_program** out) {
  if (!out || nreg < 1 || !circuits || !observables) return fail(QS_EINVAL, "bad arguments");
  *out = nullptr;
  qs_batch_program* P = new qs_batch_program();
  const int rc = build_program(nreg, circuits, observables, tile_qubits, P);
  if (rc != QS_OK) {
    const std::string msg = qs_last_error();
    free_program(P);
    return fail(rc, "%s", msg.c_str());
  }
  *out = P;
  return QS_OK;
}

int qs_batch_program_create_ex(int nreg, const qs_circuit* const* circuits, const qs_observable* const* observables,
                               int tile_qubits, int phase_qubits, int flags, qs_batch_program** out) {
  if (!out || nreg < 1 || !circuits || !observables) return fail(QS_EINVAL, "bad arguments");
  if (flags & ~QS_BATCH_PRECISE) return fail(QS_EINVAL, "unknown program flags 0x%x", flags);
  *out = nullptr;
  qs_batch_program* P = new qs_batch_program();
  const bool precise = (flags & QS_BATCH_PRECISE) != 0;
  const int rb = phase_qubits > 0 ? phase_qubits : (precise ? 3 : kRB);  // the widest phase of the path
  const int rc = build_program(nreg, circuits, observables, tile_qubits, P, rb, precise);
  if (rc != QS_OK) {
    const std::string msg = qs_last_error();
    free_program(P);
    return fail(rc, "%s", msg.c_str());
  }
  *out = P;
  return QS_OK;
}

int qs_batch_program_shape(const qs_batch_program* p, int* tile_qubits, int* phase_qubits, int* flags) {
  if (!p) return fail(QS_EINVAL, "null program");
  if (tile_qubits) *tile_qubits = p->tile;
  if (phase_qubits) *phase_qubits = p->rb;
  if (flags) *flags = p->precise ? QS_BATCH_PRECISE : 0;
  return QS_OK;
}

int qs_batch_autotune_ex(int nreg, const qs_circuit* const* circuits, const qs_observable* const* observables,
                         int flags, qs_state* s, const double* dev_params, double* dev_loss, double* dev_grad,
                         int reps, int* best_tile, int* best_phase, int* ncand, int32_t* host_tiles,
                         int32_t* host_phases, double* host_ms) {
  if (!circuits || !observables || !s || !dev_params || !dev_loss || !best_tile || !best_phase)
    return fail(QS_EINVAL, "null argument");
  if (flags & ~QS_BATCH_PRECISE) return fail(QS_EINVAL, "unknown program flags 0x%x", flags);
  if (reps < 1) reps = 1;
  const bool precise = (flags & QS_BATCH_PRECISE) != 0;
  const int rflags = QS_BATCH_RESET | (dev_grad ? QS_BATCH_GRAD : 0);
  int best = -1, bestrb = -1, nc = 0;
  double best_ms = 0;
  cudaEvent_t e0, e1;
  QS_CUDA(cudaEventCreate(&e0));
  QS_CUDA(cudaEventCreate(&e1));
  int rc = QS_OK;
  for (int rb = precise ? 3 : kRB; rb >= kMinRB && rc == QS_OK; --rb) {
    const int mt = max_tile(rb);
    for (int m = mt; m >= std::max(kRowBits + rb + 2, mt - 2) && rc == QS_OK; --m) {
      qs_batch_program* P = nullptr;
      double ms = -1;
      const int crc = qs_batch_program_create_ex(nreg, circuits, observables, m, rb, flags, &P);
      if (crc == QS_OK) {
        rc = qs_batch_run(s, P, dev_params, dev_loss, dev_grad, rflags);  // warm-up
        if (rc == QS_OK && cudaEventRecord(e0, s->stream) != cudaSuccess) rc = fail(QS_EDEVICE, "event record");
        for (int r = 0; r < reps && rc == QS_OK; ++r) rc = qs_batch_run(s, P, dev_params, dev_loss, dev_grad, rflags);
        if (rc == QS_OK && cudaEventRecord(e1, s->stream) != cudaSuccess) rc = fail(QS_EDEVICE, "event record");
        if (rc == QS_OK && cudaEventSynchronize(e1) != cudaSuccess) rc = fail(QS_EDEVICE, "event sync");
        float t = 0;
        if (rc == QS_OK && cudaEventElapsedTime(&t, e0, e1) == cudaSuccess) ms = (double)t / reps;
        qs_batch_program_destroy(P);
      } else if (crc != QS_EUNSUPPORTED && crc != QS_EINVAL) {
        rc = crc;
      }
      if (ncand && nc < *ncand) {
        if (host_tiles) host_tiles[nc] = m;
        if (host_phases) host_phases[nc] = rb;
        if (host_ms) host_ms[nc] = ms;
      }
      ++nc;
      if (ms >= 0 && (best < 0 || ms < best_ms)) {
        best = m;
        bestrb = rb;
        best_ms = ms;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != QS_OK) return rc;
  if (ncand) *ncand = nc;
  if (best < 0) return fail(QS_EUNSUPPORTED, "no program shape ran the batch");
  *best_tile = best;
  *best_phase = bestrb;
  return QS_OK;
}

int qs_batch_program_destroy(qs_batch_program* p) {
  free_program(p);
  return QS_OK;
}

int qs_batch_program_info(const qs_batch_program* p, int* nreg, int64_t* nparams_total, int64_t* host_param_offsets,
                          int64_t* host_amp_offsets) {
  if (!p) return fail(QS_EINVAL, "null program");
  if (nreg) *nreg = p->nreg;
  if (nparams_total) *nparams_total = p->param_off[p->nreg];
  if (host_param_offsets) std::copy(p->param_off.begin(), p->param_off.end(), host_param_offsets);
  if (host_amp_offsets) std::copy(p->amp_off.begin(), p->amp_off.end(), host_amp_offsets);
  return QS_OK;
}

int qs_batch_run(qs_state* s, const qs_batch_program* p, const double* dev_params, double* dev_loss,
                 double* dev_grad, int flags) {
  if (!s || !p || !dev_loss) return fail(QS_EINVAL, "null argument");
  if (s->dtype != QS_C64) return fail(QS_EUNSUPPORTED, "the batched engine runs complex64 states");
  if (s->nreg != p->nreg) return fail(QS_EINVAL, "state has %d registers, program %d", s->nreg, p->nreg);
  for (int r = 0; r < s->nreg; ++r)
    if (s->nq[r] != p->nq[r]) return fail(QS_EINVAL, "register %d: %d qubits in the state, %d in the program", r, s->nq[r], p->nq[r]);
  if (p->param_off[p->nreg] > 0 && !dev_params) return fail(QS_EINVAL, "params is NULL");
  const bool grad = (flags & QS_BATCH_GRAD) != 0;
  if (grad && !dev_grad) return fail(QS_EINVAL, "grad is NULL");
  int dev = 0;
  QS_CUDA(cudaGetDevice(&dev));
  if (dev != p->device)
    return fail(QS_EINVAL, "the program was built on device %d; the current device is %d", p->device, dev);
  cudaStream_t st = s->stream;
  QS_TRY(launch_prep(p, dev_params, true, st));
  QS_CUDA(cudaMemsetAsync(p->counter, 0, sizeof(int), st));
  BArgs a;
  a.state = (float2*)s->data;
  a.dtab = p->dtab;
  a.druns = p->druns;
  a.wpsi = p->wpsi;
  a.wlam = p->wlam;
  a.wpsif = p->wpsif;
  a.wlamf = p->wlamf;
  a.flo = p->flo;
  a.blo = p->blo;
  a.dtlo = p->dtlo;
  a.regs = p->regs;
  a.order = p->order;
  a.passes = p->passes;
  a.phases = p->phases;
  a.fops = p->fops;
  a.bops = p->bops;
  a.terms = p->terms;
  a.loss = dev_loss;
  a.grad = dev_grad;
  a.counter = p->counter;
  a.nreg = p->nreg;
  a.flags = ((flags & QS_BATCH_RESET) ? BF_RESET : 0) | (grad ? BF_GRAD : 0);
  if (p->precise) {
    if (p->rb == 2) k_batch<2, true><<<p->blocks, kTileThreads, p->smem, st>>>(a);
    else k_batch<3, true><<<p->blocks, kTileThreads, p->smem, st>>>(a);
  } else {
    switch (p->rb) {
      case 2: k_batch<2, false><<<p->blocks, kTileThreads, p->smem, st>>>(a); break;
      case 3: k_batch<3, false><<<p->blocks, kTileThreads, p->smem, st>>>(a); break;
      default: k_batch<4, false><<<p->blocks, kTileThreads, p->smem, st>>>(a); break;
    }
  }
  QS_LAUNCHED();
  return QS_OK;
}

}  // extern "C"
