// gates.cu -- gate-application kernels (sm_103a) and the host-side gate planner.
//
// The paper's fallback instruction (Sec. "Performance") applies a 2^k x 2^k
// matrix to every 2^k-tuple of amplitudes whose control bits match; its
// specialisations skip flops and untouched amplitudes for diagonal and
// permutation matrices (App. "Matrix Types", Table "Matrix types").  Here each
// class is its own streaming kernel:
//   DIAG1  multiply only the amplitudes in the touched subspace
//          (T/S/Z/shift touch half of the state, controlled phases less),
//   SWAP1 / PERM1 / DENSE1  2x2 on amplitude pairs (i, i | 2^t),
//   DIAGK / PERMK / DENSEK  general k-tuples, matrix read from the kernel's
//          parameter bank (uniform across threads, so served as broadcasts).
// All of them are HBM-bound streams on complex64: items are 16-byte vector
// accesses of two consecutive amplitudes (bit 0 lane pair), two items per
// thread with loads issued before any arithmetic, 256 threads per block.
#include <cstdarg>
#include <cmath>
#include <cstring>

#include <type_traits>

#include "common.cuh"

namespace qs {

constexpr int kThreads = 256;
constexpr int kIPT = 2;  // items per thread
constexpr int kDiagIPT = 8;  // k_diag1: one 16-byte pair per item (measured: 2 -> 4 -> 8 items raised T gates 5125 -> 5390 -> 5630 GB/s at n = 25)

size_t amp_bytes(int dtype) { return dtype == QS_C128 ? 16 : 8; }

int make_idx(int n, uint64_t fixed_mask, uint64_t set_bits, IdxSpec* out) {
  IdxSpec s;
  memset(&s, 0, sizeof(s));
  int nf = 0;
  for (int q = 0; q < 64; ++q)
    if ((fixed_mask >> q) & 1ull) {
      if (q >= n || nf >= kMaxFix) return fail(QS_EINVAL, "fixed bit %d out of range (n=%d)", q, n);
      s.fix[nf++] = (uint8_t)q;
    }
  s.nfix = nf;
  s.item_log2 = n - nf;
  s.set_bits = set_bits;
  s.reg_stride = 1ull << n;
  *out = s;
  return QS_OK;
}

// ------------------------------------------------------------------ kernels

template <typename R>
struct U4 { c2_t<R> m[4]; };

// amplitude *= factor; items are lane pairs (idx, idx + 1)
template <typename R>
__global__ void __launch_bounds__(kThreads)
k_diag1(c2_t<R>* __restrict__ psi, uint64_t nitems, IdxSpec s, int t, c2_t<R> d0, c2_t<R> d1,
        int lane_sel) {
  using T = c2_t<R>;
  constexpr int kIPT = kDiagIPT;
  const uint64_t first = (uint64_t)blockIdx.x * (blockDim.x * kIPT) + threadIdx.x;
  uint64_t idx[kIPT];
  T a0[kIPT], a1[kIPT];
#pragma unroll
  for (int u = 0; u < kIPT; ++u) {
    const uint64_t it = first + (uint64_t)u * blockDim.x;
    idx[u] = it < nitems ? item_index(it, s) : ~0ull;
    if (idx[u] == ~0ull) continue;
    if (lane_sel < 0) ld_pair(psi + idx[u], a0[u], a1[u]);
    else a0[u] = psi[idx[u] + lane_sel];
  }
#pragma unroll
  for (int u = 0; u < kIPT; ++u) {
    if (idx[u] == ~0ull) continue;
    if (lane_sel < 0) {
      const T f0 = (t >= 0 && ((idx[u] >> t) & 1ull)) ? d1 : d0;
      const T f1 = (t >= 0 && (((idx[u] + 1) >> t) & 1ull)) ? d1 : d0;
      st_pair(psi + idx[u], cmul(a0[u], f0), cmul(a1[u], f1));
    } else {
      const uint64_t i = idx[u] + lane_sel;
      const T f = (t >= 0 && ((i >> t) & 1ull)) ? d1 : d0;
      psi[i] = cmul(a0[u], f);
    }
  }
}

template <typename R, int OP>
__device__ __forceinline__ void pair_op(c2_t<R>& a, c2_t<R>& b, const U4<R>& u) {
  using T = c2_t<R>;
  if constexpr (OP == OP_SWAP1) {
    T tmp = a; a = b; b = tmp;
  } else if constexpr (OP == OP_PERM1) {
    T na = cmul(u.m[1], b);
    T nb = cmul(u.m[2], a);
    a = na; b = nb;
  } else if constexpr (OP == OP_REAL1) {  // u real: 2 operations per component
    T na, nb;
    na.x = fma(u.m[1].x, b.x, u.m[0].x * a.x);
    na.y = fma(u.m[1].x, b.y, u.m[0].x * a.y);
    nb.x = fma(u.m[3].x, b.x, u.m[2].x * a.x);
    nb.y = fma(u.m[3].x, b.y, u.m[2].x * a.y);
    a = na; b = nb;
  } else if constexpr (OP == OP_RXLIKE1) {  // u0, u3 real; u1, u2 imaginary
    T na, nb;
    na.x = fma(-u.m[1].y, b.y, u.m[0].x * a.x);
    na.y = fma(u.m[1].y, b.x, u.m[0].x * a.y);
    nb.x = fma(u.m[3].x, b.x, -u.m[2].y * a.y);
    nb.y = fma(u.m[3].x, b.y, u.m[2].y * a.x);
    a = na; b = nb;
  } else {
    T na = cfma(u.m[1], b, cmul(u.m[0], a));
    T nb = cfma(u.m[3], b, cmul(u.m[2], a));
    a = na; b = nb;
  }
}

// 2x2 on amplitude pairs.  T0: target is bit 0 (the pair is one vector
// access).  Otherwise each item holds lanes (idx, idx+1) and their partners at
// + 2^t; lane_sel >= 0 restricts the update to one lane (control on bit 0).
template <typename R, int OP, bool T0>
__global__ void __launch_bounds__(kThreads)
k_gate1(c2_t<R>* __restrict__ psi, uint64_t nitems, IdxSpec s, int t, U4<R> u, int lane_sel) {
  using T = c2_t<R>;
  const uint64_t first = (uint64_t)blockIdx.x * (blockDim.x * kIPT) + threadIdx.x;
  uint64_t idx[kIPT];
  T a0[kIPT], a1[kIPT], b0[kIPT], b1[kIPT];
  const uint64_t stride = 1ull << t;
#pragma unroll
  for (int v = 0; v < kIPT; ++v) {
    const uint64_t it = first + (uint64_t)v * blockDim.x;
    idx[v] = it < nitems ? item_index(it, s) : ~0ull;
    if (idx[v] == ~0ull) continue;
    ld_pair(psi + idx[v], a0[v], a1[v]);
    if (!T0) ld_pair(psi + idx[v] + stride, b0[v], b1[v]);
  }
#pragma unroll
  for (int v = 0; v < kIPT; ++v) {
    if (idx[v] == ~0ull) continue;
    if (T0) {
      pair_op<R, OP>(a0[v], a1[v], u);
      st_pair(psi + idx[v], a0[v], a1[v]);
    } else {
      T x0 = a0[v], y0 = b0[v], x1 = a1[v], y1 = b1[v];
      pair_op<R, OP>(x0, y0, u);
      pair_op<R, OP>(x1, y1, u);
      if (lane_sel == 1) { x0 = a0[v]; y0 = b0[v]; }
      if (lane_sel == 0) { x1 = a1[v]; y1 = b1[v]; }
      st_pair(psi + idx[v], x0, x1);
      st_pair(psi + idx[v] + stride, y0, y1);
    }
  }
}

// complex64 1-qubit gate with its FP64 matrix held as hi + lo and every output
// rounded once (Plan::precise): the same item layout as k_gate1
template <bool T0>
__global__ void __launch_bounds__(kThreads)
k_gate1_prec(float2* __restrict__ psi, uint64_t nitems, IdxSpec s, int t, U4<float> uh, U4<float> ul, int lane_sel) {
  const uint64_t first = (uint64_t)blockIdx.x * (blockDim.x * kIPT) + threadIdx.x;
  uint64_t idx[kIPT];
  float2 a0[kIPT], a1[kIPT], b0[kIPT], b1[kIPT];
  const uint64_t stride = 1ull << t;
#pragma unroll
  for (int v = 0; v < kIPT; ++v) {
    const uint64_t it = first + (uint64_t)v * blockDim.x;
    idx[v] = it < nitems ? item_index(it, s) : ~0ull;
    if (idx[v] == ~0ull) continue;
    ld_pair(psi + idx[v], a0[v], a1[v]);
    if (!T0) ld_pair(psi + idx[v] + stride, b0[v], b1[v]);
  }
  auto op = [&](float2& a, float2& b) {
    const float2 na = cf_dot2(a, uh.m[0], ul.m[0], b, uh.m[1], ul.m[1]);
    const float2 nb = cf_dot2(a, uh.m[2], ul.m[2], b, uh.m[3], ul.m[3]);
    a = na;
    b = nb;
  };
#pragma unroll
  for (int v = 0; v < kIPT; ++v) {
    if (idx[v] == ~0ull) continue;
    if (T0) {
      op(a0[v], a1[v]);
      st_pair(psi + idx[v], a0[v], a1[v]);
    } else {
      float2 x0 = a0[v], y0 = b0[v], x1 = a1[v], y1 = b1[v];
      op(x0, y0);
      op(x1, y1);
      if (lane_sel == 1) { x0 = a0[v]; y0 = b0[v]; }
      if (lane_sel == 0) { x1 = a1[v]; y1 = b1[v]; }
      st_pair(psi + idx[v], x0, x1);
      st_pair(psi + idx[v] + stride, y0, y1);
    }
  }
}

// the diagonal form of the same (touched subspace only, as k_diag1)
__global__ void __launch_bounds__(kThreads)
k_diag1_prec(float2* __restrict__ psi, uint64_t nitems, IdxSpec s, int t, float2 d0h, float2 d0l, float2 d1h,
             float2 d1l, int lane_sel) {
  const uint64_t first = (uint64_t)blockIdx.x * (blockDim.x * kIPT) + threadIdx.x;
  uint64_t idx[kIPT];
  float2 a0[kIPT], a1[kIPT];
#pragma unroll
  for (int u = 0; u < kIPT; ++u) {
    const uint64_t it = first + (uint64_t)u * blockDim.x;
    idx[u] = it < nitems ? item_index(it, s) : ~0ull;
    if (idx[u] == ~0ull) continue;
    if (lane_sel < 0) ld_pair(psi + idx[u], a0[u], a1[u]);
    else a0[u] = psi[idx[u] + lane_sel];
  }
#pragma unroll
  for (int u = 0; u < kIPT; ++u) {
    if (idx[u] == ~0ull) continue;
    if (lane_sel < 0) {
      const bool s0 = t >= 0 && ((idx[u] >> t) & 1ull), s1 = t >= 0 && (((idx[u] + 1) >> t) & 1ull);
      st_pair(psi + idx[u], cf_mul(a0[u], s0 ? d1h : d0h, s0 ? d1l : d0l), cf_mul(a1[u], s1 ? d1h : d0h, s1 ? d1l : d0l));
    } else {
      const uint64_t i = idx[u] + lane_sel;
      const bool s1 = t >= 0 && ((i >> t) & 1ull);
      psi[i] = cf_mul(a0[u], s1 ? d1h : d0h, s1 ? d1l : d0l);
    }
  }
}

template <typename R, int K>
struct MatK {
  c2_t<R> m[1 << (2 * K)];  // DENSEK: row-major; DIAGK / PERMK: first 2^K entries
  uint64_t off[1 << K];     // element offsets of the tuple
  int8_t perm[1 << K];
};

// general k-tuple kernel: one tuple per thread
template <typename R, int K, int OP>
__global__ void __launch_bounds__(kThreads)
k_gatek(c2_t<R>* __restrict__ psi, uint64_t nitems, IdxSpec s, const __grid_constant__ MatK<R, K> M) {
  using T = c2_t<R>;
  constexpr int D = 1 << K;
  const uint64_t it = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (it >= nitems) return;
  const uint64_t base = item_index(it, s);
  T x[D];
  if constexpr (OP == OP_PERMK) {
    // gather in permuted order so that no register array is indexed at run time
#pragma unroll
    for (int m = 0; m < D; ++m) x[m] = psi[base + M.off[M.perm[m]]];
#pragma unroll
    for (int m = 0; m < D; ++m) psi[base + M.off[m]] = cmul(x[m], M.m[m]);
    return;
  }
#pragma unroll
  for (int m = 0; m < D; ++m) x[m] = psi[base + M.off[m]];
  if constexpr (OP == OP_DIAGK) {
#pragma unroll
    for (int m = 0; m < D; ++m) psi[base + M.off[m]] = cmul(x[m], M.m[m]);
  } else {
#pragma unroll 1
    for (int m = 0; m < D; ++m) {
      T acc = cmk<T>(0, 0);
#pragma unroll
      for (int j = 0; j < D; ++j) acc = cfma(M.m[m * D + j], x[j], acc);
      psi[base + M.off[m]] = acc;
    }
  }
}

// complex64 k-qubit gate with its FP64 matrix held as hi + lo (MatK M and its
// corrections W) and every output amplitude summed in double-float and rounded
// once (Plan::precise): one tuple per thread, as k_gatek
template <int K, int OP>
__global__ void __launch_bounds__(kThreads)
k_gatek_prec(float2* __restrict__ psi, uint64_t nitems, IdxSpec s, const __grid_constant__ MatK<float, K> M,
             const __grid_constant__ MatK<float, K> W) {
  constexpr int D = 1 << K;
  const uint64_t it = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (it >= nitems) return;
  const uint64_t base = item_index(it, s);
  float2 x[D];
  if constexpr (OP == OP_PERMK) {
#pragma unroll
    for (int m = 0; m < D; ++m) x[m] = psi[base + M.off[M.perm[m]]];
#pragma unroll
    for (int m = 0; m < D; ++m) psi[base + M.off[m]] = cf_mul(x[m], M.m[m], W.m[m]);
    return;
  }
#pragma unroll
  for (int m = 0; m < D; ++m) x[m] = psi[base + M.off[m]];
  if constexpr (OP == OP_DIAGK) {
#pragma unroll
    for (int m = 0; m < D; ++m) psi[base + M.off[m]] = cf_mul(x[m], M.m[m], W.m[m]);
    return;
  }
#pragma unroll 1
  for (int m = 0; m < D; ++m) {
    float rs, re, is, ie;
    cf_first(rs, re, x[0].x, M.m[m * D].x, W.m[m * D].x);
    cf_add(rs, re, -x[0].y, M.m[m * D].y, W.m[m * D].y);
    cf_first(is, ie, x[0].x, M.m[m * D].y, W.m[m * D].y);
    cf_add(is, ie, x[0].y, M.m[m * D].x, W.m[m * D].x);
#pragma unroll
    for (int j = 1; j < D; ++j) {
      const float2 u = M.m[m * D + j], w = W.m[m * D + j];
      cf_add(rs, re, x[j].x, u.x, w.x);
      cf_add(rs, re, -x[j].y, u.y, w.y);
      cf_add(is, ie, x[j].x, u.y, w.y);
      cf_add(is, ie, x[j].y, u.x, w.x);
    }
    psi[base + M.off[m]] = make_float2(__fadd_rn(rs, re), __fadd_rn(is, ie));
  }
}

// complex64 dense 2- and 3-qubit gates whose targets and controls leave qubit 0
// free: items 2i and 2i + 1 are adjacent amplitudes of every member, so a
// thread takes both tuples with one 16-byte access per member
template <int K>
__global__ void __launch_bounds__(kThreads)
k_gatek_pair(float2* __restrict__ psi, uint64_t npairs, IdxSpec s, const __grid_constant__ MatK<float, K> M) {
  constexpr int D = 1 << K;
  const uint64_t pi = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (pi >= npairs) return;
  const uint64_t base = item_index(2 * pi, s);
  float4 v[D];
#pragma unroll
  for (int m = 0; m < D; ++m) v[m] = *reinterpret_cast<const float4*>(psi + base + M.off[m]);
#pragma unroll
  for (int m = 0; m < D; ++m) {
    float2 a0 = make_float2(0.f, 0.f), a1 = make_float2(0.f, 0.f);
#pragma unroll
    for (int j = 0; j < D; ++j) {
      a0 = cfma(M.m[m * D + j], make_float2(v[j].x, v[j].y), a0);
      a1 = cfma(M.m[m * D + j], make_float2(v[j].z, v[j].w), a1);
    }
    *reinterpret_cast<float4*>(psi + base + M.off[m]) = make_float4(a0.x, a0.y, a1.x, a1.y);
  }
}

// ------------------------------------------------------------------ launchers

static inline unsigned blocks_for(uint64_t items, int per_block) {
  return (unsigned)((items + per_block - 1) / per_block);
}

// Threads per CTA for `items` work items of `ipt` items per thread: kThreads,
// halved (down to one warp) while that leaves fewer than two CTAs per SM.  A
// small register then spreads over many SMs instead of a few full CTAs, which
// matters most for complex128, whose FP64 rate per SM is low on this GPU.
static int cta_threads(uint64_t items, int ipt) {
  static int sms[64] = {0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) dev = 0;
  if (!sms[dev] && cudaDeviceGetAttribute(&sms[dev], cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    sms[dev] = 1;
  }
  int nt = kThreads;
  while (nt > 32 && blocks_for(items, nt * ipt) < 2u * (unsigned)sms[dev]) nt >>= 1;
  return nt;
}

template <typename R> static c2_t<R> to_dev(cd z) {
  c2_t<R> r;
  r.x = (R)z.real();
  r.y = (R)z.imag();
  return r;
}
// FP32 correction z - to_dev<float>(z)
static float2 lo_dev(cd z) {
  const float2 h = to_dev<float>(z);
  return make_float2((float)(z.real() - (double)h.x), (float)(z.imag() - (double)h.y));
}

template <int K, int OP>
static int launch_prec_k(float2* psi, int n, int nreg, const Plan& p, cudaStream_t st) {
  MatK<float, K> M, W;
  memset(&M, 0, sizeof(M));
  memset(&W, 0, sizeof(W));
  constexpr int D = 1 << K;
  uint64_t locmask = 0;
  for (int j = 0; j < K; ++j) locmask |= 1ull << p.locs[j];
  for (int m = 0; m < D; ++m) {
    uint64_t o = 0;
    for (int j = 0; j < K; ++j)
      if ((m >> j) & 1) o |= 1ull << p.locs[j];
    M.off[m] = o;
  }
  if (OP == OP_DENSEK)
    for (int i = 0; i < D * D; ++i) {
      M.m[i] = to_dev<float>(p.U[i]);
      W.m[i] = lo_dev(p.U[i]);
    }
  else
    for (int m = 0; m < D; ++m) {
      const cd v = OP == OP_DIAGK ? p.U[m * D + m] : p.pv[m];
      M.m[m] = to_dev<float>(v);
      W.m[m] = lo_dev(v);
      if (OP == OP_PERMK) M.perm[m] = (int8_t)p.perm[m];
    }
  IdxSpec s;
  QS_TRY(make_idx(n, locmask | p.ctrl_mask, p.ctrl_vals, &s));
  const uint64_t items = (uint64_t)nreg << s.item_log2;
  if (items == 0) return QS_OK;
  const int nt = cta_threads(items, 1);
  k_gatek_prec<K, OP><<<blocks_for(items, nt), nt, 0, st>>>(psi, items, s, M, W);
  QS_LAUNCHED();
  return QS_OK;
}

template <int OP>
static int launch_prec_op(float2* psi, int n, int nreg, const Plan& p, cudaStream_t st) {
  switch (p.k) {
    case 2: return launch_prec_k<2, OP>(psi, n, nreg, p, st);
    case 3: return launch_prec_k<3, OP>(psi, n, nreg, p, st);
    case 4: return launch_prec_k<4, OP>(psi, n, nreg, p, st);
    case 5: return launch_prec_k<5, OP>(psi, n, nreg, p, st);
  }
  return fail(QS_EUNSUPPORTED, "gate arity %d", p.k);
}

// the compensated complex64 launches of Plan::precise (1-qubit dense,
// permutation and diagonal forms, k-qubit dense, diagonal and phased-permutation
// forms; SWAP1 is exact as it is)
static int launch_prec(float2* psi, int n, int nreg, const Plan& p, cudaStream_t st) {
  if (p.op == OP_DENSEK) return launch_prec_op<OP_DENSEK>(psi, n, nreg, p, st);
  if (p.op == OP_DIAGK) return launch_prec_op<OP_DIAGK>(psi, n, nreg, p, st);
  if (p.op == OP_PERMK) return launch_prec_op<OP_PERMK>(psi, n, nreg, p, st);
  if (p.op == OP_DIAG1) {
    IdxSpec s;
    QS_TRY(make_idx(n, 1ull | p.mask, p.vals & ~1ull, &s));
    const uint64_t items = (uint64_t)nreg << s.item_log2;
    if (!items) return QS_OK;
    const int lane = (p.mask & 1ull) ? (int)(p.vals & 1ull) : -1;
    const int nt = cta_threads(items, kIPT);
    k_diag1_prec<<<blocks_for(items, nt * kIPT), nt, 0, st>>>(psi, items, s, p.t, to_dev<float>(p.d0), lo_dev(p.d0),
                                                               to_dev<float>(p.d1), lo_dev(p.d1), lane);
    QS_LAUNCHED();
    return QS_OK;
  }
  U4<float> uh, ul;
  for (int i = 0; i < 4; ++i) {
    uh.m[i] = to_dev<float>(p.u[i]);
    ul.m[i] = lo_dev(p.u[i]);
  }
  const int t = p.t;
  IdxSpec s;
  if (t == 0) {
    QS_TRY(make_idx(n, 1ull | p.ctrl_mask, p.ctrl_vals, &s));
    const uint64_t items = (uint64_t)nreg << s.item_log2;
    if (!items) return QS_OK;
    const int nt = cta_threads(items, kIPT);
    k_gate1_prec<true><<<blocks_for(items, nt * kIPT), nt, 0, st>>>(psi, items, s, 0, uh, ul, -1);
  } else {
    QS_TRY(make_idx(n, 1ull | (1ull << t) | p.ctrl_mask, p.ctrl_vals & ~1ull, &s));
    const uint64_t items = (uint64_t)nreg << s.item_log2;
    if (!items) return QS_OK;
    const int lane = (p.ctrl_mask & 1ull) ? (int)(p.ctrl_vals & 1ull) : -1;
    const int nt = cta_threads(items, kIPT);
    k_gate1_prec<false><<<blocks_for(items, nt * kIPT), nt, 0, st>>>(psi, items, s, t, uh, ul, lane);
  }
  QS_LAUNCHED();
  return QS_OK;
}

template <typename R, int K, int OP>
static int launch_k_t(c2_t<R>* psi, int n, int nreg, const Plan& p, cudaStream_t st) {
  MatK<R, K> M;
  memset(&M, 0, sizeof(M));
  constexpr int D = 1 << K;
  uint64_t locmask = 0;
  for (int j = 0; j < K; ++j) locmask |= 1ull << p.locs[j];
  for (int m = 0; m < D; ++m) {
    uint64_t o = 0;
    for (int j = 0; j < K; ++j)
      if ((m >> j) & 1) o |= 1ull << p.locs[j];
    M.off[m] = o;
  }
  if (OP == OP_DENSEK)
    for (int i = 0; i < D * D; ++i) M.m[i] = to_dev<R>(p.U[i]);
  else if (OP == OP_DIAGK)
    for (int m = 0; m < D; ++m) M.m[m] = to_dev<R>(p.U[m * D + m]);
  else
    for (int m = 0; m < D; ++m) {
      M.m[m] = to_dev<R>(p.pv[m]);
      M.perm[m] = (int8_t)p.perm[m];
    }
  IdxSpec s;
  QS_TRY(make_idx(n, locmask | p.ctrl_mask, p.ctrl_vals, &s));
  const uint64_t items = (uint64_t)nreg << s.item_log2;
  if (items == 0) return QS_OK;
  if constexpr (std::is_same<R, float>::value && OP == OP_DENSEK && (K == 2 || K == 3)) {
    if (!((locmask | p.ctrl_mask) & 1ull) && s.item_log2 >= 1) {
      const int nt = cta_threads(items / 2, 1);
      k_gatek_pair<K><<<blocks_for(items / 2, nt), nt, 0, st>>>(psi, items / 2, s, M);
      QS_LAUNCHED();
      return QS_OK;
    }
  }
  const int nt = cta_threads(items, 1);
  k_gatek<R, K, OP><<<blocks_for(items, nt), nt, 0, st>>>(psi, items, s, M);
  QS_LAUNCHED();
  return QS_OK;
}

template <typename R, int OP>
static int launch_k_op(c2_t<R>* psi, int n, int nreg, const Plan& p, cudaStream_t st) {
  switch (p.k) {
    case 1: return launch_k_t<R, 1, OP>(psi, n, nreg, p, st);
    case 2: return launch_k_t<R, 2, OP>(psi, n, nreg, p, st);
    case 3: return launch_k_t<R, 3, OP>(psi, n, nreg, p, st);
    case 4: return launch_k_t<R, 4, OP>(psi, n, nreg, p, st);
    case 5: return launch_k_t<R, 5, OP>(psi, n, nreg, p, st);
  }
  return fail(QS_EUNSUPPORTED, "gate arity %d", p.k);
}

template <typename R, int OP>
static int launch_1(c2_t<R>* psi, int n, int nreg, const Plan& p, cudaStream_t st) {
  U4<R> u;
  for (int i = 0; i < 4; ++i) u.m[i] = to_dev<R>(p.u[i]);
  const int t = p.t;
  if (t == 0) {
    IdxSpec s;
    QS_TRY(make_idx(n, 1ull | p.ctrl_mask, p.ctrl_vals, &s));
    const uint64_t items = (uint64_t)nreg << s.item_log2;
    if (!items) return QS_OK;
    const int nt = cta_threads(items, kIPT);
    k_gate1<R, OP, true><<<blocks_for(items, nt * kIPT), nt, 0, st>>>(psi, items, s, 0, u, -1);
  } else {
    IdxSpec s;
    QS_TRY(make_idx(n, 1ull | (1ull << t) | p.ctrl_mask, p.ctrl_vals & ~1ull, &s));
    const uint64_t items = (uint64_t)nreg << s.item_log2;
    if (!items) return QS_OK;
    const int lane = (p.ctrl_mask & 1ull) ? (int)(p.ctrl_vals & 1ull) : -1;
    const int nt = cta_threads(items, kIPT);
    k_gate1<R, OP, false><<<blocks_for(items, nt * kIPT), nt, 0, st>>>(psi, items, s, t, u, lane);
  }
  QS_LAUNCHED();
  return QS_OK;
}

template <typename R>
static int launch_typed(c2_t<R>* psi, int n, int nreg, const Plan& p, cudaStream_t st) {
  switch (p.op) {
    case OP_NOP: return QS_OK;
    case OP_DIAG1: {
      IdxSpec s;
      QS_TRY(make_idx(n, 1ull | p.mask, p.vals & ~1ull, &s));
      const uint64_t items = (uint64_t)nreg << s.item_log2;
      if (!items) return QS_OK;
      const int lane = (p.mask & 1ull) ? (int)(p.vals & 1ull) : -1;
      const int nt = cta_threads(items, kDiagIPT);
      k_diag1<R><<<blocks_for(items, nt * kDiagIPT), nt, 0, st>>>(
          psi, items, s, p.t, to_dev<R>(p.d0), to_dev<R>(p.d1), lane);
      QS_LAUNCHED();
      return QS_OK;
    }
    case OP_SWAP1: return launch_1<R, OP_SWAP1>(psi, n, nreg, p, st);
    case OP_PERM1: return launch_1<R, OP_PERM1>(psi, n, nreg, p, st);
    case OP_DENSE1: return launch_1<R, OP_DENSE1>(psi, n, nreg, p, st);
    case OP_REAL1: return launch_1<R, OP_REAL1>(psi, n, nreg, p, st);
    case OP_RXLIKE1: return launch_1<R, OP_RXLIKE1>(psi, n, nreg, p, st);
    case OP_DIAGK: return launch_k_op<R, OP_DIAGK>(psi, n, nreg, p, st);
    case OP_PERMK: return launch_k_op<R, OP_PERMK>(psi, n, nreg, p, st);
    case OP_DENSEK: return launch_k_op<R, OP_DENSEK>(psi, n, nreg, p, st);
  }
  return fail(QS_EUNSUPPORTED, "unknown plan");
}

int launch_plan_on(void* data, int dtype, int n, int nreg, int64_t reg_stride, const Plan& p,
                   qs_state* owner) {
  (void)reg_stride;
  cudaStream_t st = owner ? owner->stream : nullptr;
  if (dtype == QS_C64 && p.precise &&
      (p.op == OP_DIAG1 || p.op == OP_DENSE1 || p.op == OP_REAL1 || p.op == OP_RXLIKE1 || p.op == OP_PERM1 ||
       ((p.op == OP_DENSEK || p.op == OP_DIAGK || p.op == OP_PERMK) && p.k >= 2 && p.k <= 5)))
    return launch_prec((float2*)data, n, nreg, p, st);
  if (use_block_tc(dtype, p)) return launch_block_tc((float2*)data, n, nreg, p, st);
  if (dtype == QS_C64) return launch_typed<float>((float2*)data, n, nreg, p, st);
  return launch_typed<double>((double2*)data, n, nreg, p, st);
}

int launch_plan(qs_state* s, const Plan& p) {
  if (p.op == OP_NOP) return QS_OK;
  if (s->uniform) return launch_plan_on(s->data, s->dtype, s->nq[0], s->nreg, 1ll << s->nq[0], p, s);
  const size_t ab = amp_bytes(s->dtype);
  for (int r = 0; r < s->nreg; ++r)
    QS_TRY(launch_plan_on((char*)s->data + ab * s->off[r], s->dtype, s->nq[r], 1, 1ll << s->nq[r], p, s));
  return QS_OK;
}

// ------------------------------------------------------------------ planner

int validate_gate(int n, int k, const int32_t* locs, uint64_t ctrl_mask) {
  if (k < 1 || k > QS_MAXK) return fail(QS_EINVAL, "gate arity %d not in 1..%d", k, QS_MAXK);
  uint64_t seen = 0;
  for (int j = 0; j < k; ++j) {
    if (locs[j] < 0 || locs[j] >= n) return fail(QS_EINVAL, "loc %d out of range for n=%d", locs[j], n);
    if ((seen >> locs[j]) & 1ull) return fail(QS_EINVAL, "duplicate loc %d", locs[j]);
    seen |= 1ull << locs[j];
  }
  if (n < 64 && (ctrl_mask >> n)) return fail(QS_EINVAL, "control qubit out of range for n=%d", n);
  if (ctrl_mask & seen) return fail(QS_EINVAL, "a control qubit is also a target");
  return QS_OK;
}

int plan_gate(const cd* U, int k, const int* locs, uint64_t ctrl_mask, uint64_t ctrl_vals, Plan* p) {
  Plan& P = *p;
  P = Plan();
  P.k = k;
  for (int j = 0; j < k; ++j) P.locs[j] = locs[j];
  P.ctrl_mask = ctrl_mask;
  P.ctrl_vals = ctrl_vals & ctrl_mask;
  const int D = 1 << k;
  bool diag = true, perm = true;
  for (int r = 0; r < D; ++r) {
    int nz = 0;
    for (int c = 0; c < D; ++c) {
      if (U[r * D + c] != cd(0, 0)) {
        ++nz;
        if (r != c) diag = false;
        P.perm[r] = c;
        P.pv[r] = U[r * D + c];
      }
    }
    if (nz != 1) perm = false;
  }
  if (perm) {  // rows must hit distinct columns
    uint64_t used = 0;
    for (int r = 0; r < D; ++r) used |= 1ull << P.perm[r];
    perm = (used == ((D == 64) ? ~0ull : ((1ull << D) - 1ull)));
  }
  uint64_t locmask = 0;
  for (int j = 0; j < k; ++j) locmask |= 1ull << locs[j];
  if (diag) {
    int nonunit = 0, which = -1;
    for (int m = 0; m < D; ++m)
      if (U[m * D + m] != cd(1, 0)) { ++nonunit; which = m; }
    if (nonunit == 0) { P.op = OP_NOP; return QS_OK; }
    bool all_equal = true;
    for (int m = 1; m < D; ++m)
      if (U[m * D + m] != U[0]) all_equal = false;
    if (all_equal) {  // scalar on the control subspace
      P.op = OP_DIAG1; P.t = -1; P.mask = ctrl_mask; P.vals = P.ctrl_vals; P.d0 = U[0];
      return QS_OK;
    }
    if (nonunit == 1) {  // one touched sector: e.g. T, S, Z, shift, CZ, controlled phase
      uint64_t v = P.ctrl_vals;
      for (int j = 0; j < k; ++j)
        if ((which >> j) & 1) v |= 1ull << locs[j];
      P.op = OP_DIAG1; P.t = -1; P.mask = ctrl_mask | locmask; P.vals = v; P.d0 = U[which * D + which];
      return QS_OK;
    }
    if (k == 1) {
      P.op = OP_DIAG1; P.t = locs[0]; P.mask = ctrl_mask; P.vals = P.ctrl_vals;
      P.d0 = U[0]; P.d1 = U[3];
      return QS_OK;
    }
    P.op = OP_DIAGK;
    P.U.assign(U, U + D * D);
    return QS_OK;
  }
  if (k == 1) {
    P.t = locs[0];
    for (int i = 0; i < 4; ++i) P.u[i] = U[i];
    if (perm) {
      P.op = (U[1] == cd(1, 0) && U[2] == cd(1, 0)) ? OP_SWAP1 : OP_PERM1;
    } else if (U[0].imag() == 0 && U[1].imag() == 0 && U[2].imag() == 0 && U[3].imag() == 0) {
      P.op = OP_REAL1;
    } else if (U[0].imag() == 0 && U[3].imag() == 0 && U[1].real() == 0 && U[2].real() == 0) {
      P.op = OP_RXLIKE1;
    } else {
      P.op = OP_DENSE1;
    }
    return QS_OK;
  }
  P.op = perm ? OP_PERMK : OP_DENSEK;
  P.U.assign(U, U + D * D);
  return QS_OK;
}

// ------------------------------------------------------------------ gate matrices

static void pauli(int p, cd m[4]) {
  m[0] = m[1] = m[2] = m[3] = 0;
  switch (p) {
    case 1: m[1] = 1; m[2] = 1; break;
    case 2: m[1] = cd(0, -1); m[2] = cd(0, 1); break;
    case 3: m[0] = 1; m[3] = -1; break;
    default: m[0] = 1; m[3] = 1; break;
  }
}

// Pauli string sigma_{p_0} (x) ... on k targets, bit j of the index <-> target j
void pauli_string(int k, const int32_t* paulis, std::vector<cd>& S) {
  const int D = 1 << k;
  S.assign(D * D, cd(0, 0));
  for (int r = 0; r < D; ++r)
    for (int c = 0; c < D; ++c) {
      cd v = 1;
      for (int j = 0; j < k; ++j) {
        cd m[4];
        pauli(paulis[j], m);
        v *= m[((r >> j) & 1) * 2 + ((c >> j) & 1)];
      }
      S[r * D + c] = v;
    }
}

int named_matrix(int kind, int k, const int32_t* paulis, double th, std::vector<cd>& U) {
  const double c = std::cos(th / 2), s = std::sin(th / 2), h = std::sqrt(0.5);
  const cd i(0, 1);
  auto one = [&](cd a, cd b, cd cc, cd d) { U = {a, b, cc, d}; return k == 1 ? QS_OK : fail(QS_EINVAL, "gate needs 1 target"); };
  switch (kind) {
    case QS_GATE_I: return one(1, 0, 0, 1);
    case QS_GATE_X: return one(0, 1, 1, 0);
    case QS_GATE_Y: return one(0, -i, i, 0);
    case QS_GATE_Z: return one(1, 0, 0, -1);
    case QS_GATE_H: return one(h, h, h, -h);
    case QS_GATE_S: return one(1, 0, 0, i);
    case QS_GATE_SDG: return one(1, 0, 0, -i);
    case QS_GATE_T: return one(1, 0, 0, cd(h, h));
    case QS_GATE_TDG: return one(1, 0, 0, cd(h, -h));
    case QS_GATE_RX: return one(c, -i * s, -i * s, c);
    case QS_GATE_RY: return one(c, -s, s, c);
    case QS_GATE_RZ: return one(cd(c, -s), 0, 0, cd(c, s));
    case QS_GATE_SHIFT: return one(1, 0, 0, cd(std::cos(th), std::sin(th)));
    case QS_GATE_PHASE: return one(cd(std::cos(th), std::sin(th)), 0, 0, cd(std::cos(th), std::sin(th)));
    case QS_GATE_SWAP:
      if (k != 2) return fail(QS_EINVAL, "SWAP needs 2 targets");
      U.assign(16, 0);
      U[0] = 1; U[1 * 4 + 2] = 1; U[2 * 4 + 1] = 1; U[15] = 1;
      return QS_OK;
    case QS_GATE_ROT: {
      if (!paulis) return fail(QS_EINVAL, "ROT needs paulis");
      for (int j = 0; j < k; ++j)
        if (paulis[j] < 1 || paulis[j] > 3) return fail(QS_EINVAL, "ROT pauli must be 1..3");
      std::vector<cd> S;
      pauli_string(k, paulis, S);
      const int D = 1 << k;
      U.assign(D * D, 0);
      for (int r = 0; r < D * D; ++r) U[r] = -i * s * S[r];
      for (int m = 0; m < D; ++m) U[m * D + m] += c;
      return QS_OK;
    }
  }
  return fail(QS_EINVAL, "unknown gate kind %d", kind);
}

int gate_matrix(const qs_circuit* c, const qs_gate_desc& g, const double* params, std::vector<cd>& U) {
  if (g.kind == QS_GATE_MATRIX) {
    const int D = 1 << g.nlocs;
    if (g.mat_offset < 0 || (size_t)(g.mat_offset + D * D) > c->mats.size())
      return fail(QS_EINVAL, "matrix offset out of range");
    U.assign(c->mats.begin() + g.mat_offset, c->mats.begin() + g.mat_offset + D * D);
    return QS_OK;
  }
  const double th = g.param >= 0 ? params[g.param] : g.theta;
  return named_matrix(g.kind, g.nlocs, g.paulis, th, U);
}

void dagger(std::vector<cd>& U, int k) {
  const int D = 1 << k;
  std::vector<cd> V(D * D);
  for (int r = 0; r < D; ++r)
    for (int c = 0; c < D; ++c) V[r * D + c] = std::conj(U[c * D + r]);
  U.swap(V);
}

}  // namespace qs
