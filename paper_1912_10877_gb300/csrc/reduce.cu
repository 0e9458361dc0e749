// reduce.cu -- expectation values, lambda = O psi, measurement sampling, reset
// and collapse (sm_103a).
//
// expect (Sec. "Forward Mode"): O = sum_t c_t P_t with P_t a Pauli string.
// For a basis state, P|i> = i^{nY} (-1)^{popc(i & z)} |i ^ x>, so
// <psi|P|psi> = sum_i ph(i) conj(psi_{i^x}) psi_i.  Terms are grouped by their
// x mask; one streaming pass per group reads each amplitude (or each pair
// (i, i^x) once, counting it twice) and accumulates every term of the group in
// FP64.  The sum is pairwise: a thread adds at most kSerialItems items in
// order (the serial base case), warps and blocks combine by balanced trees,
// and a second kernel folds the per-block partials of every term by a
// balanced tree as well (fixed shapes, so results are reproducible run to
// run).  Error bound: (kSerialItems + log2 of the item count) * 2^-53 of the
// sum of the absolute terms.
//
// measure (Sec. "Instructions on Quantum Registers"): the deterministic
// contract of qsim.h -- FP64 probabilities with separately rounded multiply
// and add, left folds over level-0 blocks of 1024 probabilities and level-1
// blocks of 1024 level-0 sums, and a three-level walk per shot.
#include <cmath>
#include <cstring>
#include <map>

#include "common.cuh"

namespace qs {

constexpr int kRedThreads = 256;
constexpr int kSerialItems = 64;  // serial base case of the pairwise expectation sums
constexpr int kGroupTerms = 16;   // terms of one x-mask group handled per launch
constexpr int kObsChunk = 64;     // terms per lambda = O psi launch

struct TermGroup {
  int nt;
  int item_log2;
  int h;                 // highest bit of x (-1 if x == 0)
  uint64_t x;
  uint64_t z[kGroupTerms];
  int ny[kGroupTerms];   // number of Y factors mod 4
};

__device__ __forceinline__ double2 ld_amp(const float2* p, uint64_t i) {
  const float2 v = p[i];
  return make_double2((double)v.x, (double)v.y);
}
__device__ __forceinline__ double2 ld_amp(const double2* p, uint64_t i) { return p[i]; }

__device__ __forceinline__ double term_value(int ny, double s, double zr, double zi) {
  switch (ny & 3) {
    case 0: return s * zr;
    case 1: return -s * zi;
    case 2: return -s * zr;
    default: return s * zi;
  }
}

// grid (blocks_per_reg, nreg); partials[(reg * nt_total + term_base + t) * nblk + block]
template <typename T>
__global__ void __launch_bounds__(kRedThreads)
k_expect_group(const T* __restrict__ psi, uint64_t reg_stride, TermGroup g, double* __restrict__ partials,
               int nt_total, int term_base) {
  const int nblk = gridDim.x;
  const uint64_t r = blockIdx.y;
  const T* p = psi + r * reg_stride;
  const uint64_t items = 1ull << g.item_log2;
  double acc[kGroupTerms];
#pragma unroll
  for (int t = 0; t < kGroupTerms; ++t) acc[t] = 0.0;
  for (uint64_t j = (uint64_t)blockIdx.x * kRedThreads + threadIdx.x; j < items;
       j += (uint64_t)nblk * kRedThreads) {
    uint64_t i = j;
    if (g.h >= 0) i = ((j >> g.h) << (g.h + 1)) | (j & ((1ull << g.h) - 1ull));
    const double2 a = ld_amp(p, i);
    double zr, zi;
    if (g.h >= 0) {
      const double2 b = ld_amp(p, i ^ g.x);
      zr = b.x * a.x + b.y * a.y;
      zi = b.x * a.y - b.y * a.x;
    } else {
      zr = a.x * a.x + a.y * a.y;
      zi = 0.0;
    }
#pragma unroll
    for (int t = 0; t < kGroupTerms; ++t) {
      if (t < g.nt) {
        const double s = (__popcll(i & g.z[t]) & 1) ? -1.0 : 1.0;
        acc[t] += term_value(g.ny[t], s, zr, zi);
      }
    }
  }
  __shared__ double red[kRedThreads / 32][kGroupTerms];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int t = 0; t < kGroupTerms; ++t) {
    double v = acc[t];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) red[warp][t] = v;
  }
  __syncthreads();
  if (threadIdx.x < g.nt) {
    static_assert(kRedThreads / 32 == 8, "block tree below is written for 8 warps");
    const int t = threadIdx.x;
    const double v = ((red[0][t] + red[1][t]) + (red[2][t] + red[3][t])) +
                     ((red[4][t] + red[5][t]) + (red[6][t] + red[7][t]));
    const double f = g.h >= 0 ? 2.0 : 1.0;
    partials[((r * nt_total) + term_base + threadIdx.x) * nblk + blockIdx.x] = f * v;
  }
}

// Pairwise sum in index order of the values add()ed one by one: a binary
// counter of partial sums, so 2^k values form a balanced tree.
struct PairwiseAcc {
  double stk[40];
  uint64_t cnt = 0;
  __device__ void add(double v) {
    int lvl = 0;
    while ((cnt >> lvl) & 1ull) {
      v = stk[lvl] + v;
      ++lvl;
    }
    stk[lvl] = v;
    ++cnt;
  }
  __device__ double total() const {
    double r = 0.0;
    bool any = false;
    for (int lvl = 0; lvl < 40; ++lvl)
      if ((cnt >> lvl) & 1ull) {
        r = any ? stk[lvl] + r : stk[lvl];
        any = true;
      }
    return r;
  }
};

constexpr int kFoldThreads = 256;

// Pairwise sum of v[0..len) by one CTA of kFoldThreads threads: contiguous
// chunks per thread (binary counter), then a shared-memory tree.  Every thread
// receives the result.
__device__ double block_pairwise(const double* __restrict__ v, int64_t len, double* sh) {
  const int64_t chunk = (len + kFoldThreads - 1) / kFoldThreads;
  const int64_t lo = (int64_t)threadIdx.x * chunk, hi = lo + chunk < len ? lo + chunk : len;
  PairwiseAcc acc;
  for (int64_t i = lo; i < hi; ++i) acc.add(v[i]);
  sh[threadIdx.x] = acc.total();
  __syncthreads();
  for (int w = kFoldThreads / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) sh[threadIdx.x] = sh[threadIdx.x] + sh[threadIdx.x + w];
    __syncthreads();
  }
  const double r = sh[0];
  __syncthreads();
  return r;
}

// one CTA per register: every term's block partials folded pairwise, then the
// terms' c_t * v_t pairwise in term order.
__global__ void __launch_bounds__(kFoldThreads)
k_expect_final(const double* __restrict__ partials, int nblk, int nt_total, const double* __restrict__ coeff,
               double* __restrict__ out) {
  __shared__ double sh[kFoldThreads];
  const int r = blockIdx.x;
  PairwiseAcc terms;
  for (int t = 0; t < nt_total; ++t) {
    const double v = block_pairwise(partials + ((size_t)r * nt_total + t) * nblk, nblk, sh);
    terms.add(coeff[t] * v);
  }
  if (threadIdx.x == 0) out[r] = terms.total();
}

// blocks per register for the pairwise expectation: at most kSerialItems items per thread
static int expect_blocks(uint64_t items) {
  const uint64_t per_block = (uint64_t)kRedThreads * kSerialItems;
  return (int)std::max<uint64_t>(1, (items + per_block - 1) / per_block);
}

struct ObsChunk {
  int nt;
  uint64_t x[kObsChunk];
  uint64_t z[kObsChunk];
  int ny[kObsChunk];
  double c[kObsChunk];
};

// lam (+)= sum_t c_t P_t psi, FP64 (complex128 buffers), one amplitude per thread
__global__ void __launch_bounds__(256)
k_apply_obs(const double2* __restrict__ psi, double2* __restrict__ lam, uint64_t dim, int accumulate,
            const __grid_constant__ ObsChunk o) {
  const uint64_t i = (uint64_t)blockIdx.x * 256 + threadIdx.x;
  if (i >= dim) return;
  double2 acc = accumulate ? lam[i] : make_double2(0.0, 0.0);
  for (int t = 0; t < o.nt; ++t) {
    const uint64_t j = i ^ o.x[t];          // (P psi)_i = ph(j) psi_j, j = i ^ x
    const double2 v = psi[j];
    const double s = (__popcll(j & o.z[t]) & 1) ? -o.c[t] : o.c[t];
    double re, im;
    switch (o.ny[t] & 3) {
      case 0: re = v.x; im = v.y; break;
      case 1: re = -v.y; im = v.x; break;   // * i
      case 2: re = -v.x; im = -v.y; break;  // * -1
      default: re = v.y; im = -v.x; break;  // * -i
    }
    acc.x += s * re;
    acc.y += s * im;
  }
  lam[i] = acc;
}

// ------------------------------------------------------------------ host side

static int grouped(const qs_observable* o, std::vector<std::pair<uint64_t, std::vector<int>>>& groups) {
  std::map<uint64_t, std::vector<int>> m;
  for (int t = 0; t < (int)o->terms.size(); ++t) m[o->terms[t].x_mask].push_back(t);
  groups.assign(m.begin(), m.end());
  return QS_OK;
}

// expectation of registers stored at `data` (uniform: nreg x 2^n, else one register)
int expect_raw(const void* data, int dtype, int n, int nreg, const qs_observable* o, qs_state* ws_owner,
               double* host_out) {
  cudaStream_t st = ws_owner->stream;
  const int nt_total = (int)o->terms.size();
  for (const auto& t : o->terms) {
    if (n < 64 && ((t.x_mask | t.z_mask) >> n)) return fail(QS_EINVAL, "observable acts on a qubit >= n=%d", n);
  }
  std::vector<std::pair<uint64_t, std::vector<int>>> groups;
  grouped(o, groups);
  const uint64_t dim = 1ull << n;
  // every group's items: 2^n (x = 0) or 2^(n-1) pairs; the grid covers the larger
  const int nblk = expect_blocks(dim);
  const size_t part_bytes = sizeof(double) * (size_t)nreg * std::max(1, nt_total) * nblk;
  const size_t coeff_off = (part_bytes + 255) / 256 * 256;
  const size_t out_off = coeff_off + (sizeof(double) * std::max(1, nt_total) + 255) / 256 * 256;
  QS_TRY(ensure_ws(ws_owner, ws_owner->ws, out_off + sizeof(double) * nreg));
  double* partials = (double*)ws_owner->ws.ptr;
  double* dcoeff = (double*)((char*)ws_owner->ws.ptr + coeff_off);
  double* dev_out = (double*)((char*)ws_owner->ws.ptr + out_off);
  // coefficients in the global term order of the partials layout below
  std::vector<double> coeff;
  std::vector<int> order;
  for (auto& g : groups)
    for (int t : g.second) { order.push_back(t); coeff.push_back(o->terms[t].coeff); }
  if (nt_total > 0)
    QS_CUDA(cudaMemcpyAsync(dcoeff, coeff.data(), sizeof(double) * nt_total, cudaMemcpyHostToDevice, st));
  int base = 0;
  for (auto& g : groups) {
    const auto& ids = g.second;
    for (size_t c0 = 0; c0 < ids.size(); c0 += kGroupTerms) {
      TermGroup tg;
      memset(&tg, 0, sizeof(tg));
      tg.x = g.first;
      tg.h = g.first ? 63 - __builtin_clzll(g.first) : -1;
      tg.item_log2 = g.first ? n - 1 : n;
      tg.nt = (int)std::min<size_t>(kGroupTerms, ids.size() - c0);
      for (int t = 0; t < tg.nt; ++t) {
        const auto& term = o->terms[ids[c0 + t]];
        tg.z[t] = term.z_mask;
        tg.ny[t] = __builtin_popcountll(term.x_mask & term.z_mask) & 3;
      }
      dim3 grid(nblk, nreg);
      if (dtype == QS_C64)
        k_expect_group<float2><<<grid, kRedThreads, 0, st>>>((const float2*)data, dim, tg, partials, nt_total, base);
      else
        k_expect_group<double2><<<grid, kRedThreads, 0, st>>>((const double2*)data, dim, tg, partials, nt_total, base);
      QS_LAUNCHED();
      base += tg.nt;
    }
  }
  if (nt_total == 0) {
    QS_CUDA(cudaMemsetAsync(dev_out, 0, sizeof(double) * nreg, st));
  } else {
    k_expect_final<<<nreg, kFoldThreads, 0, st>>>(partials, nblk, nt_total, dcoeff, dev_out);
    QS_LAUNCHED();
  }
  QS_CUDA(cudaMemcpyAsync(host_out, dev_out, sizeof(double) * nreg, cudaMemcpyDeviceToHost, st));
  QS_CUDA(cudaStreamSynchronize(st));
  return QS_OK;
}

int apply_observable_c128(const double2* psi, double2* lam, int n, const qs_observable* o, cudaStream_t st) {
  const uint64_t dim = 1ull << n;
  const int nt = (int)o->terms.size();
  if (nt == 0) {
    QS_CUDA(cudaMemsetAsync(lam, 0, sizeof(double2) * dim, st));
    return QS_OK;
  }
  for (int c0 = 0; c0 < nt; c0 += kObsChunk) {
    ObsChunk ch;
    memset(&ch, 0, sizeof(ch));
    ch.nt = std::min(kObsChunk, nt - c0);
    for (int t = 0; t < ch.nt; ++t) {
      const auto& term = o->terms[c0 + t];
      ch.x[t] = term.x_mask;
      ch.z[t] = term.z_mask;
      ch.ny[t] = __builtin_popcountll(term.x_mask & term.z_mask) & 3;
      ch.c[t] = term.coeff;
    }
    k_apply_obs<<<(unsigned)((dim + 255) / 256), 256, 0, st>>>(psi, lam, dim, c0 > 0, ch);
    QS_LAUNCHED();
  }
  return QS_OK;
}

// ------------------------------------------------------------------ sampling

constexpr int kF = 1024;

template <typename T>
__device__ __forceinline__ double prob(const T* p, uint64_t i) {
  const double2 a = ld_amp(p, i);
  return __dadd_rn(__dmul_rn(a.x, a.x), __dmul_rn(a.y, a.y));
}

template <typename T>
__global__ void k_level0(const T* __restrict__ psi, uint64_t dim, uint64_t nb0, double* __restrict__ s0) {
  const uint64_t b = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nb0) return;
  const uint64_t lo = b * kF, hi = lo + kF < dim ? lo + kF : dim;
  double a = prob(psi, lo);
  for (uint64_t i = lo + 1; i < hi; ++i) a = __dadd_rn(a, prob(psi, i));
  s0[b] = a;
}

__global__ void k_level1(const double* __restrict__ s0, uint64_t nb0, uint64_t nb1, double* __restrict__ s1) {
  const uint64_t c = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= nb1) return;
  const uint64_t lo = c * kF, hi = lo + kF < nb0 ? lo + kF : nb0;
  double a = s0[lo];
  for (uint64_t b = lo + 1; b < hi; ++b) a = __dadd_rn(a, s0[b]);
  s1[c] = a;
}

// the walk of the contract: first j whose running sum exceeds t, else the last
// positive value, else the last; acc carries the exclusive prefix
template <typename F>
__device__ uint64_t walk(F value, uint64_t len, double t, double& acc) {
  double a = acc, a_last = acc;
  int64_t last = -1;
  for (uint64_t j = 0; j < len; ++j) {
    const double v = value(j);
    const double nxt = __dadd_rn(a, v);
    if (nxt > t) { acc = a; return j; }
    if (v > 0.0) { last = (int64_t)j; a_last = a; }
    a = nxt;
  }
  if (last >= 0) { acc = a_last; return (uint64_t)last; }
  return len - 1;
}

template <typename T>
__global__ void k_sample(const T* __restrict__ psi, uint64_t dim, const double* __restrict__ s0, uint64_t nb0,
                         const double* __restrict__ s1, uint64_t nb1, const double* __restrict__ u, int nshots,
                         int64_t* __restrict__ out) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= nshots) return;
  double total = s1[0];
  for (uint64_t c = 1; c < nb1; ++c) total = __dadd_rn(total, s1[c]);
  const double t = __dmul_rn(u[s], total);
  double acc = 0.0;
  const uint64_t c = walk([&](uint64_t j) { return s1[j]; }, nb1, t, acc);
  const uint64_t b0 = c * kF, b1 = b0 + kF < nb0 ? b0 + kF : nb0;
  const uint64_t b = b0 + walk([&](uint64_t j) { return s0[b0 + j]; }, b1 - b0, t, acc);
  const uint64_t i0 = b * kF, i1 = i0 + kF < dim ? i0 + kF : dim;
  out[s] = (int64_t)(i0 + walk([&](uint64_t j) { return prob(psi, i0 + j); }, i1 - i0, t, acc));
}

template <typename T>
__global__ void k_collapse_scale(T* psi, int64_t x, double2* keep) {
  const double2 a = ld_amp(psi, (uint64_t)x);
  const double r = sqrt(a.x * a.x + a.y * a.y);
  *keep = r > 0.0 ? make_double2(a.x / r, a.y / r) : make_double2(1.0, 0.0);
}

__device__ __forceinline__ void st_amp(float2* p, uint64_t i, double2 v) { p[i] = make_float2((float)v.x, (float)v.y); }
__device__ __forceinline__ void st_amp(double2* p, uint64_t i, double2 v) { p[i] = v; }

template <typename T>
__global__ void k_collapse_write(T* psi, uint64_t dim, int64_t x, const double2* keep) {
  const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= dim) return;
  st_amp(psi, i, i == (uint64_t)x ? *keep : make_double2(0.0, 0.0));
}

// one register at `data` with 2^n amplitudes
// samples of one register with device uniforms into device indices; scratch:
// sample_scratch_doubles(n) doubles (block sums of the three-level walk)
size_t sample_scratch_doubles(int n) {
  const uint64_t dim = 1ull << n;
  const uint64_t nb0 = (dim + kF - 1) / kF, nb1 = (nb0 + kF - 1) / kF;
  return (size_t)(nb0 + nb1);
}

int sample_dev(const void* data, int dtype, int n, const double* dev_u, int nshots, int64_t* dev_out,
               double* scratch, cudaStream_t st) {
  const uint64_t dim = 1ull << n;
  const uint64_t nb0 = (dim + kF - 1) / kF, nb1 = (nb0 + kF - 1) / kF;
  double* s0 = scratch;
  double* s1 = s0 + nb0;
  if (dtype == QS_C64) k_level0<float2><<<(unsigned)((nb0 + 127) / 128), 128, 0, st>>>((const float2*)data, dim, nb0, s0);
  else k_level0<double2><<<(unsigned)((nb0 + 127) / 128), 128, 0, st>>>((const double2*)data, dim, nb0, s0);
  QS_LAUNCHED();
  k_level1<<<(unsigned)((nb1 + 127) / 128), 128, 0, st>>>(s0, nb0, nb1, s1);
  QS_LAUNCHED();
  if (dtype == QS_C64)
    k_sample<float2><<<(nshots + 127) / 128, 128, 0, st>>>((const float2*)data, dim, s0, nb0, s1, nb1, dev_u, nshots, dev_out);
  else
    k_sample<double2><<<(nshots + 127) / 128, 128, 0, st>>>((const double2*)data, dim, s0, nb0, s1, nb1, dev_u, nshots, dev_out);
  QS_LAUNCHED();
  return QS_OK;
}

// Uniforms of the seeded measurement: draw k of SplitMix64 started from `seed`
// (Steele, Lea and Flood 2014): state seed + k * 0x9E3779B97F4A7C15, then the
// 64-bit finaliser (xor-shift 30, multiply, xor-shift 27, multiply, xor-shift
// 31); u = top 53 bits / 2^53.  Shot j of this call is draw k0 + j + 1.
__global__ void k_seeded_uniforms(uint64_t seed, uint64_t k0, int nshots, double* __restrict__ u) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= nshots) return;
  uint64_t x = seed + (k0 + (uint64_t)j + 1ull) * 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  x ^= x >> 31;
  u[j] = (double)(x >> 11) * 0x1.0p-53;
}

int measure_one(void* data, int dtype, int n, const double* host_u, int nshots, int64_t* host_out,
                int collapse, qs_state* owner, const uint64_t* seed, uint64_t k0) {
  cudaStream_t st = owner->stream;
  const uint64_t dim = 1ull << n;
  const uint64_t nb0 = (dim + kF - 1) / kF, nb1 = (nb0 + kF - 1) / kF;
  const size_t need = sizeof(double) * (nb0 + nb1) + sizeof(double) * nshots + sizeof(int64_t) * nshots + 64;
  QS_TRY(ensure_ws(owner, owner->ws, need + 256));
  char* w = (char*)owner->ws.ptr;
  double* s0 = (double*)w;
  double* s1 = s0 + nb0;
  double* du = s1 + nb1;
  int64_t* dout = (int64_t*)(du + nshots);
  double2* keep = (double2*)(((uintptr_t)(dout + nshots) + 15) & ~(uintptr_t)15);
  if (seed) {
    k_seeded_uniforms<<<(nshots + 127) / 128, 128, 0, st>>>(*seed, k0, nshots, du);
    QS_LAUNCHED();
  } else {
    QS_CUDA(cudaMemcpyAsync(du, host_u, sizeof(double) * nshots, cudaMemcpyHostToDevice, st));
  }
  if (dtype == QS_C64) {
    k_level0<float2><<<(unsigned)((nb0 + 127) / 128), 128, 0, st>>>((const float2*)data, dim, nb0, s0);
  } else {
    k_level0<double2><<<(unsigned)((nb0 + 127) / 128), 128, 0, st>>>((const double2*)data, dim, nb0, s0);
  }
  QS_LAUNCHED();
  k_level1<<<(unsigned)((nb1 + 127) / 128), 128, 0, st>>>(s0, nb0, nb1, s1);
  QS_LAUNCHED();
  if (dtype == QS_C64)
    k_sample<float2><<<(nshots + 127) / 128, 128, 0, st>>>((const float2*)data, dim, s0, nb0, s1, nb1, du, nshots, dout);
  else
    k_sample<double2><<<(nshots + 127) / 128, 128, 0, st>>>((const double2*)data, dim, s0, nb0, s1, nb1, du, nshots, dout);
  QS_LAUNCHED();
  QS_CUDA(cudaMemcpyAsync(host_out, dout, sizeof(int64_t) * nshots, cudaMemcpyDeviceToHost, st));
  QS_CUDA(cudaStreamSynchronize(st));
  if (collapse) {
    const int64_t x = host_out[0];
    if (dtype == QS_C64) {
      k_collapse_scale<float2><<<1, 1, 0, st>>>((float2*)data, x, keep);
      k_collapse_write<float2><<<(unsigned)((dim + 255) / 256), 256, 0, st>>>((float2*)data, dim, x, keep);
    } else {
      k_collapse_scale<double2><<<1, 1, 0, st>>>((double2*)data, x, keep);
      k_collapse_write<double2><<<(unsigned)((dim + 255) / 256), 256, 0, st>>>((double2*)data, dim, x, keep);
    }
    QS_LAUNCHED();
    QS_CUDA(cudaStreamSynchronize(st));
  }
  return QS_OK;
}

// ------------------------------------------------------------------ reset / promote

__global__ void k_set_ones(char* data, int dtype, const int64_t* __restrict__ pos, int count) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= count) return;
  if (dtype == QS_C64) ((float2*)data)[pos[r]] = make_float2(1.f, 0.f);
  else ((double2*)data)[pos[r]] = make_double2(1.0, 0.0);
}

int reset_basis(qs_state* s, const uint64_t* host_basis) {
  cudaStream_t st = s->stream;
  std::vector<int64_t> pos(s->nreg);
  for (int r = 0; r < s->nreg; ++r) {
    const uint64_t x = host_basis ? host_basis[r] : 0;
    if (s->nq[r] < 64 && (x >> s->nq[r])) return fail(QS_EINVAL, "basis index %llu out of range for register %d",
                                                     (unsigned long long)x, r);
    pos[r] = s->off[r] + (int64_t)x;
  }
  QS_TRY(ensure_ws(s, s->ws, sizeof(int64_t) * s->nreg));
  QS_CUDA(cudaMemsetAsync(s->data, 0, s->bytes, st));
  QS_CUDA(cudaMemcpyAsync(s->ws.ptr, pos.data(), sizeof(int64_t) * s->nreg, cudaMemcpyHostToDevice, st));
  k_set_ones<<<(s->nreg + 127) / 128, 128, 0, st>>>((char*)s->data, s->dtype, (const int64_t*)s->ws.ptr, s->nreg);
  QS_LAUNCHED();
  return QS_OK;
}

__global__ void k_promote(const float2* __restrict__ in, double2* __restrict__ out, uint64_t dim) {
  const uint64_t i = (uint64_t)blockIdx.x * 256 + threadIdx.x;
  if (i >= dim) return;
  const float2 v = in[i];
  out[i] = make_double2((double)v.x, (double)v.y);
}

int promote_to_c128(const void* in, int dtype, double2* out, uint64_t dim, cudaStream_t st) {
  if (dtype == QS_C128) {
    QS_CUDA(cudaMemcpyAsync(out, in, sizeof(double2) * dim, cudaMemcpyDeviceToDevice, st));
    return QS_OK;
  }
  k_promote<<<(unsigned)((dim + 255) / 256), 256, 0, st>>>((const float2*)in, out, dim);
  QS_LAUNCHED();
  return QS_OK;
}

}  // namespace qs

// ------------------------------------------------------------------ expectation without allocation
//
// qs_expect_static: the expectation reduction above with its scratch in a
// fixed, file-scope device array instead of memory obtained from cudaMalloc,
// for callers that cannot allocate device memory.  Every GPU that loads the
// library holds this array (512 KiB) until the process exits.  All calls
// share it, so calls whose kernels overlap on the GPU race on it.

namespace qs {

constexpr int kStaticPartials = 1 << 16;  // FP64 partial sums (512 KiB)
constexpr int kStaticTerms = 64;
constexpr int kStaticMaxDevices = 64;

static __device__ __align__(256) double g_static_partials[kStaticPartials];

struct StaticCoeffs {
  double c[kStaticTerms];
};

__global__ void __launch_bounds__(kFoldThreads)
k_expect_final_static(const double* __restrict__ partials, int nblk, int nt_total,
                      const __grid_constant__ StaticCoeffs co, double* __restrict__ out) {
  __shared__ double sh[kFoldThreads];
  const int r = blockIdx.x;
  PairwiseAcc terms;
  for (int t = 0; t < nt_total; ++t) {
    const double v = block_pairwise(partials + ((size_t)r * nt_total + t) * nblk, nblk, sh);
    terms.add(co.c[t] * v);
  }
  if (threadIdx.x == 0) out[r] = terms.total();
}

// device address of g_static_partials on the current device, resolved once per
// device (host code must not use the symbol's host-side name as an address)
static double* g_static_addr[kStaticMaxDevices];

static int static_partials(double** out) {
  int dev = 0;
  QS_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kStaticMaxDevices) return fail(QS_EUNSUPPORTED, "device ordinal %d >= %d", dev, kStaticMaxDevices);
  if (!g_static_addr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_static_partials);
    if (e != cudaSuccess || !p)
      return fail(QS_EDEVICE, "cudaGetSymbolAddress of the static scratch failed: %s", cudaGetErrorString(e));
    g_static_addr[dev] = (double*)p;
  }
  *out = g_static_addr[dev];
  return QS_OK;
}

}  // namespace qs

extern "C" int qs_expect_static(const void* dev_amps, int dtype, int nqubits, int nreg, const qs_pauli_term* host_terms,
                                int nterms, double* dev_out, void* stream) {
  using namespace qs;
  if (!dev_amps || !dev_out || (nterms > 0 && !host_terms)) return fail(QS_EINVAL, "null argument");
  if (dtype != QS_C64 && dtype != QS_C128) return fail(QS_EINVAL, "dtype must be QS_C64 or QS_C128");
  if (((uintptr_t)dev_amps % amp_bytes(dtype)) || ((uintptr_t)dev_out % sizeof(double)))
    return fail(QS_EINVAL, "misaligned amplitude or output pointer");
  if (nqubits < 1 || nqubits > QS_MAXQ) return fail(QS_EINVAL, "nqubits %d not in 1..%d", nqubits, QS_MAXQ);
  if (nreg < 1 || nreg > 65535) return fail(QS_EINVAL, "nreg %d not in 1..65535", nreg);
  if (nterms < 0 || nterms > kStaticTerms)
    return fail(QS_EINVAL, "nterms %d exceeds the static limit of %d terms", nterms, kStaticTerms);
  if ((long long)nreg * nterms > kStaticPartials)
    return fail(QS_EINVAL, "nreg * nterms = %lld exceeds the static scratch of %d partial sums",
                (long long)nreg * nterms, kStaticPartials);
  for (int t = 0; t < nterms; ++t)
    if (nqubits < 64 && ((host_terms[t].x_mask | host_terms[t].z_mask) >> nqubits))
      return fail(QS_EINVAL, "term %d acts on a qubit >= n=%d", t, nqubits);
  cudaStream_t st = (cudaStream_t)stream;
  if (nterms == 0) {
    QS_CUDA(cudaMemsetAsync(dev_out, 0, sizeof(double) * nreg, st));
    return QS_OK;
  }
  double* partials = nullptr;
  QS_TRY(static_partials(&partials));
  int cur_dev = 0;
  cudaGetDevice(&cur_dev);
  // terms ordered by x mask (insertion sort on the stack, stable)
  int order[kStaticTerms];
  for (int t = 0; t < nterms; ++t) {
    int j = t;
    while (j > 0 && host_terms[order[j - 1]].x_mask > host_terms[t].x_mask) {
      order[j] = order[j - 1];
      --j;
    }
    order[j] = t;
  }
  const uint64_t dim = 1ull << nqubits;
  long long nblk = expect_blocks(dim);
  nblk = std::max(1LL, std::min(nblk, (long long)kStaticPartials / ((long long)nreg * nterms)));
  StaticCoeffs co;
  memset(&co, 0, sizeof(co));
  int base = 0;
  while (base < nterms) {
    const uint64_t x = host_terms[order[base]].x_mask;
    TermGroup tg;
    memset(&tg, 0, sizeof(tg));
    tg.x = x;
    tg.h = x ? 63 - __builtin_clzll(x) : -1;
    tg.item_log2 = x ? nqubits - 1 : nqubits;
    while (base + tg.nt < nterms && tg.nt < kGroupTerms && host_terms[order[base + tg.nt]].x_mask == x) {
      const qs_pauli_term& term = host_terms[order[base + tg.nt]];
      tg.z[tg.nt] = term.z_mask;
      tg.ny[tg.nt] = __builtin_popcountll(term.x_mask & term.z_mask) & 3;
      co.c[base + tg.nt] = term.coeff;
      ++tg.nt;
    }
    dim3 grid((unsigned)nblk, nreg);
    if (dtype == QS_C64)
      k_expect_group<float2><<<grid, kRedThreads, 0, st>>>((const float2*)dev_amps, dim, tg, partials, nterms, base);
    else
      k_expect_group<double2><<<grid, kRedThreads, 0, st>>>((const double2*)dev_amps, dim, tg, partials, nterms, base);
    QS_LAUNCHED();
    base += tg.nt;
  }
  k_expect_final_static<<<nreg, kFoldThreads, 0, st>>>(partials, (int)nblk, nterms, co, dev_out);
  if (cudaPeekAtLastError() != cudaSuccess) g_static_addr[cur_dev] = nullptr;  // resolve again next call
  QS_LAUNCHED();
  return QS_OK;
}
