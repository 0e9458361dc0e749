// onelaunch.cu -- a whole circuit (and a diagonal expectation) on a small
// register in ONE kernel launch (sm_103a).
//
// Small registers are launch-bound: the n = 12 complex128 variational circuit
// is 55 fused 3-qubit blocks of ~2^9 tuples each, and even replayed from a CUDA
// graph every launch costs more than its arithmetic.  Here the circuit's fused
// blocks (Sec. "Performance": the general k-qubit instruction, with Sec.
// "Matrix Representation": a chain's matrix is the product of its gates') run
// back to back inside one cooperative launch over every SM: block b reads the
// state from one buffer and writes the other (each output amplitude of a tuple
// is one work item, a row of the block matrix times the tuple), and a grid
// barrier separates consecutive blocks.  complex128 arithmetic is FP64, whose
// rate per SM is low on this GPU, so the rows of one tuple are spread over
// threads (and SMs) instead of one thread doing the whole 2^k x 2^k product.
// An optional diagonal observable (sums of Z strings, Sec. "Forward Mode")
// is evaluated in the same launch: per-CTA FP64 partials, then one CTA folds
// them pairwise.
//
// The grid barrier is an arrival counter and a generation word in global
// memory.  Every CTA of a cooperative launch is resident, so it completes;
// still, each wait is bounded (iteration and wall-clock limits), after which
// the CTA raises an error flag and every CTA leaves the kernel at its next
// barrier; the library's device status word records it and qs_state_sync
// reports QS_ETIMEDOUT.
#include <cstring>
#include <vector>

#include "common.cuh"

namespace qs {

constexpr int kOLThreads = 256;
constexpr int kOLMaxTerms = 64;

struct OLBlock {
  IdxSpec spec;              // tuple bases: the block's qubits fixed to 0
  uint32_t off[1 << QS_MAXK];  // member offsets of a tuple
  int32_t k;                 // block width
  int32_t mat;               // offset (entries) of its 2^k x 2^k matrix
  int32_t group;             // tuples a CTA takes at a time
  int32_t pad;
  uint64_t ntuples;
};

struct OLSync {
  unsigned count;
  unsigned gen;
  int error;
};

struct OLArgs {
  void* psi;                 // the register (2^n amplitudes)
  void* tmp;                 // a second buffer of the same size
  const OLBlock* blocks;
  const void* mats;
  int nblocks;
  uint64_t dim;
  OLSync* sync;
  int* status;               // the library's device status word (qs_state_sync reports it)
  double* partials;          // [gridDim.x] when an observable is given
  double* out;               // <O> (device)
  int nterm;
  double coeff[kOLMaxTerms];
  uint64_t z[kOLMaxTerms];
};

__device__ __forceinline__ uint64_t ol_clock() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// all CTAs arrive; returns false (for every CTA) once any wait has given up
__device__ bool ol_barrier(OLSync* s, int* status, unsigned& gen) {
  __syncthreads();
  __shared__ int ok;
  if (threadIdx.x == 0) {
    const unsigned g = gen;
    __threadfence();
    if (atomicAdd(&s->count, 1u) == gridDim.x - 1) {
      atomicExch(&s->count, 0u);
      __threadfence();
      atomicExch(&s->gen, g + 1u);
    } else {
      const uint64_t t0 = ol_clock();
      long spins = 0;
      while (atomicAdd(&s->gen, 0u) == g) {
        if (++spins > (1l << 24) || ol_clock() - t0 > 2000000000ull || atomicAdd(&s->error, 0) != 0) {
          atomicExch(&s->error, 1);
          atomicExch(status, 1);
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
    ok = atomicAdd(&s->error, 0) == 0;
  }
  __syncthreads();
  ++gen;
  return ok != 0;
}

// one block: a CTA takes G tuples at a time (G = B.group); every output row of
// a tuple is computed by kOLSplit threads, each summing a quarter of the row's
// products, in different warps: one warp keeps only its own SM sub-partition's
// FP64 unit busy, and a row split over four warps uses all four.  Thread
// (lt, s, r) loads member r of local tuple lt (s = 0) into shared memory,
// sums the products j = s (mod kOLSplit) of row r, and the s = 0 thread adds
// the four partial sums and stores the row.  G is chosen on the host so that
// the block's tuples spread over every CTA before they fill one.
constexpr int kOLSplit = 4;

template <typename T, int K>
__device__ __forceinline__ void ol_block(const OLBlock& B, const T* __restrict__ M, const T* src, T* dst,
                                         T* xs, T* ps) {
  constexpr int D = 1 << K;
  constexpr int S = D >= kOLSplit ? kOLSplit : D;   // partial sums per row
  constexpr int TPT = S * D;                         // threads per tuple
  constexpr int J = D / S;                           // products per thread
  const int G = B.group;
  const int lt = (int)threadIdx.x / TPT, rem = (int)threadIdx.x % TPT;
  const int r = rem & (D - 1), sp = rem >> K;
  const bool active = lt < G;
  const uint32_t offr = B.off[r];
  T row[J];
  if (active) {
#pragma unroll
    for (int q = 0; q < J; ++q) row[q] = __ldg(M + r * D + sp + q * S);
  }
  for (uint64_t t0 = (uint64_t)blockIdx.x * G; t0 < B.ntuples; t0 += (uint64_t)gridDim.x * G) {
    const uint64_t t = t0 + lt;
    const bool on = active && t < B.ntuples;
    const uint64_t base = on ? item_index(t, B.spec) : 0;
    // state loads bypass L1 (ld.global.cg): a buffer read two blocks ago may
    // still sit in this SM's L1 while other SMs have rewritten it since
    if (on && sp == 0) xs[lt * D + r] = __ldcg(src + base + offr);
    __syncthreads();
    if (on) {
      const T* x = xs + lt * D;
      T acc = cmk<T>(0, 0);
#pragma unroll
      for (int q = 0; q < J; ++q) acc = cfma(row[q], x[sp + q * S], acc);
      ps[threadIdx.x] = acc;
    }
    __syncthreads();
    if (on && sp == 0) {
      T sum = ps[threadIdx.x];
#pragma unroll
      for (int q = 1; q < S; ++q) {
        const T v = ps[threadIdx.x + q * D];
        sum.x += v.x;
        sum.y += v.y;
      }
      dst[base + offr] = sum;
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(kOLThreads) k_onelaunch(const __grid_constant__ OLArgs a) {
  T* src = reinterpret_cast<T*>(a.psi);
  T* dst = reinterpret_cast<T*>(a.tmp);
  const T* mats = reinterpret_cast<const T*>(a.mats);
  unsigned gen = 0;
  const uint64_t gtid = (uint64_t)threadIdx.x * gridDim.x + blockIdx.x;  // CTA-interleaved work items
  const uint64_t gstride = (uint64_t)gridDim.x * blockDim.x;
  __shared__ T xs[kOLThreads];
  __shared__ T ps[kOLThreads];
  for (int b = 0; b < a.nblocks; ++b) {
    const OLBlock& B = a.blocks[b];
    const T* M = mats + B.mat;
    switch (B.k) {
      case 1: ol_block<T, 1>(B, M, src, dst, xs, ps); break;
      case 2: ol_block<T, 2>(B, M, src, dst, xs, ps); break;
      case 3: ol_block<T, 3>(B, M, src, dst, xs, ps); break;
      case 4: ol_block<T, 4>(B, M, src, dst, xs, ps); break;
      default: ol_block<T, 5>(B, M, src, dst, xs, ps); break;
    }
    if (!ol_barrier(a.sync, a.status, gen)) return;
    T* w = src;
    src = dst;
    dst = w;
  }
  // the result is in src: bring it to the register's buffer when it ended in the other
  if (src != reinterpret_cast<T*>(a.psi)) {
    for (uint64_t i = gtid; i < a.dim; i += gstride) dst[i] = __ldcg(src + i);
    if (!ol_barrier(a.sync, a.status, gen)) return;
    src = dst;
  }
  if (a.nterm <= 0) return;
  // <O> for O = sum_t c_t Z-string_t: per-thread FP64 sums, warp and CTA trees
  double e = 0.0;
  for (uint64_t i = gtid; i < a.dim; i += gstride) {
    double w = 0.0;
    for (int t = 0; t < a.nterm; ++t) w += (__popcll(i & a.z[t]) & 1) ? -a.coeff[t] : a.coeff[t];
    const T v = __ldcg(src + i);
    e += w * ((double)v.x * (double)v.x + (double)v.y * (double)v.y);
  }
  for (int o = 16; o > 0; o >>= 1) e += __shfl_xor_sync(0xffffffffu, e, o);
  __shared__ double red[kOLThreads / 32];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = e;
  __syncthreads();
  if (threadIdx.x == 0) {
    static_assert(kOLThreads / 32 == 8, "CTA tree below is written for 8 warps");
    a.partials[blockIdx.x] = ((red[0] + red[1]) + (red[2] + red[3])) + ((red[4] + red[5]) + (red[6] + red[7]));
  }
  if (!ol_barrier(a.sync, a.status, gen)) return;
  if (blockIdx.x == 0) {
    // pairwise over the CTA partials (gridDim.x <= 2 x kOLThreads)
    __shared__ double buf[2 * kOLThreads];
    for (int i = threadIdx.x; i < 2 * kOLThreads; i += blockDim.x) buf[i] = i < (int)gridDim.x ? __ldcg(a.partials + i) : 0.0;
    __syncthreads();
    for (int w = kOLThreads; w > 0; w >>= 1) {
      for (int i = threadIdx.x; i < w; i += blockDim.x) buf[i] = buf[i] + buf[i + w];
      __syncthreads();
    }
    if (threadIdx.x == 0) *a.out = buf[0];
  }
}

// device tables of one circuit's blocks for one block width, dtype, device and
// parameter vector
struct OLCache {
  int kmax = 0, dtype = -1, device = -1, nb = 0;
  std::vector<double> params;
  std::vector<OLBlock> host_blocks;   // group fields set per launch
  OLBlock* blocks = nullptr;          // device copy (rewritten when the groups change)
  void* mats = nullptr;
  int grid = -1;
};

void free_onelaunch(const qs_circuit* c) {
  OLCache* k = static_cast<OLCache*>(c->onelaunch);
  if (!k) return;
  int cur = -1;
  const bool swap = k->device >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != k->device &&
                    cudaSetDevice(k->device) == cudaSuccess;
  if (k->blocks) cudaFree(k->blocks);
  if (k->mats) cudaFree(k->mats);
  if (swap) cudaSetDevice(cur);
  delete k;
  c->onelaunch = nullptr;
}

// the circuit's blocks (matrices formed on the host) as device tables, reused
// while the width, dtype, device and parameters stay the same
static int onelaunch_tables(qs_state* s, const qs_circuit* c, const double* host_params, int kmax, OLCache** out) {
  int dev = 0;
  QS_CUDA(cudaGetDevice(&dev));
  OLCache* k = static_cast<OLCache*>(c->onelaunch);
  const int np = c->nparams;
  if (k && k->kmax == kmax && k->dtype == s->dtype && k->device == dev && (int)k->params.size() == np &&
      (np == 0 || std::memcmp(k->params.data(), host_params, sizeof(double) * np) == 0)) {
    *out = k;
    return QS_OK;
  }
  free_onelaunch(c);
  const int n = c->nqubits;
  int nb = 0;
  QS_TRY(qs_circuit_blocks(c, host_params, kmax, &nb, nullptr, nullptr, nullptr));
  std::vector<int32_t> widths(std::max(1, nb)), locs((size_t)std::max(1, nb) * QS_MAXK);
  const size_t stride = (size_t)1 << (2 * QS_MAXK);
  std::vector<double> mats((size_t)2 * stride * std::max(1, nb));
  QS_TRY(qs_circuit_blocks(c, host_params, kmax, &nb, widths.data(), locs.data(), mats.data()));
  const size_t ab = amp_bytes(s->dtype);
  std::vector<OLBlock> blocks(nb);
  std::vector<unsigned char> pool;
  for (int b = 0; b < nb; ++b) {
    OLBlock& B = blocks[b];
    memset(&B, 0, sizeof(B));
    const int w = widths[b], D = 1 << w;
    if (w > QS_MAXK) return fail(QS_EUNSUPPORTED, "a gate spans more than %d qubits", QS_MAXK);
    uint64_t mask = 0;
    for (int j = 0; j < w; ++j) mask |= 1ull << locs[b * QS_MAXK + j];
    QS_TRY(make_idx(n, mask, 0, &B.spec));
    for (int m = 0; m < D; ++m) {
      uint32_t off = 0;
      for (int j = 0; j < w; ++j)
        if ((m >> j) & 1) off |= 1u << locs[b * QS_MAXK + j];
      B.off[m] = off;
    }
    B.k = w;
    B.ntuples = 1ull << (n - w);
    B.mat = (int32_t)(pool.size() / ab);
    const double* M = mats.data() + 2 * stride * b;
    const size_t at = pool.size();
    pool.resize(at + ab * (size_t)D * D);
    for (int i = 0; i < D * D; ++i) {
      if (s->dtype == QS_C128) {
        const double2 v = make_double2(M[2 * i], M[2 * i + 1]);
        std::memcpy(pool.data() + at + ab * i, &v, sizeof(v));
      } else {
        const float2 v = make_float2((float)M[2 * i], (float)M[2 * i + 1]);
        std::memcpy(pool.data() + at + ab * i, &v, sizeof(v));
      }
    }
  }
  k = new OLCache();
  k->kmax = kmax;
  k->dtype = s->dtype;
  k->device = dev;
  k->nb = nb;
  k->params.assign(host_params ? host_params : nullptr, host_params ? host_params + np : nullptr);
  k->host_blocks = blocks;
  c->onelaunch = k;  // owned by the circuit from here (freed with it)
  if (cudaMalloc((void**)&k->blocks, sizeof(OLBlock) * std::max(1, nb)) != cudaSuccess ||
      cudaMalloc(&k->mats, std::max<size_t>(16, pool.size())) != cudaSuccess) {
    cudaGetLastError();
    free_onelaunch(c);
    return fail(QS_ENOMEM, "cudaMalloc of the one-launch tables failed");
  }
  if (!pool.empty()) QS_CUDA(cudaMemcpy(k->mats, pool.data(), pool.size(), cudaMemcpyHostToDevice));
  *out = k;
  return QS_OK;
}

}  // namespace qs

using namespace qs;

extern "C" {

int qs_run_circuit_one_launch(qs_state* s, const qs_circuit* c, const double* host_params, int kmax,
                              const qs_observable* o, int grid_ctas, double* dev_out) {
  if (!s || !c) return fail(QS_EINVAL, "null argument");
  if (s->nreg != 1 || s->nq[0] != c->nqubits) return fail(QS_EINVAL, "one register of the circuit's size");
  if (c->nparams > 0 && !host_params) return fail(QS_EINVAL, "params is NULL");
  if (kmax < 1 || kmax > QS_MAXK) return fail(QS_EINVAL, "block width %d not in 1..%d", kmax, QS_MAXK);
  if (o && !dev_out) return fail(QS_EINVAL, "dev_out is NULL");
  const int n = s->nq[0];
  if (n > 24) return fail(QS_EUNSUPPORTED, "the one-launch path is for small registers (n <= 24)");
  OLArgs a;
  memset(&a, 0, sizeof(a));
  if (o) {
    if ((int)o->terms.size() > kOLMaxTerms) return fail(QS_EUNSUPPORTED, "more than %d observable terms", kOLMaxTerms);
    for (const auto& t : o->terms) {
      if (t.x_mask) return fail(QS_EUNSUPPORTED, "the one-launch expectation takes diagonal observables (Z strings)");
      if (n < 64 && (t.z_mask >> n)) return fail(QS_EINVAL, "observable qubit out of range");
      a.coeff[a.nterm] = t.coeff;
      a.z[a.nterm] = t.z_mask;
      ++a.nterm;
    }
  }
  OLCache* k = nullptr;
  QS_TRY(onelaunch_tables(s, c, host_params, kmax, &k));
  const int nb = k->nb;
  const size_t ab = amp_bytes(s->dtype);
  // grid: every SM (or the caller's count), all CTAs resident (cooperative launch)
  static int sms_of[64] = {0}, per_sm_of[2][64] = {{0}};
  int dev = 0;
  QS_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return fail(QS_EUNSUPPORTED, "device ordinal %d", dev);
  const void* fn = s->dtype == QS_C128 ? (const void*)k_onelaunch<double2> : (const void*)k_onelaunch<float2>;
  if (!sms_of[dev]) {
    int coop = 0;
    QS_CUDA(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
    if (!coop) return fail(QS_EUNSUPPORTED, "the device has no cooperative launch");
    QS_CUDA(cudaDeviceGetAttribute(&sms_of[dev], cudaDevAttrMultiProcessorCount, dev));
  }
  int& per_sm = per_sm_of[s->dtype == QS_C128 ? 1 : 0][dev];
  if (!per_sm) QS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kOLThreads, 0));
  const int sms = sms_of[dev];
  const int max_grid = std::min(sms * std::max(1, per_sm), 2 * kOLThreads);
  const int grid = grid_ctas > 0 ? std::min(grid_ctas, max_grid) : std::min(sms, max_grid);
  cudaStream_t st = s->stream;
  if (k->grid != grid) {
    // tuples per CTA at a time: as many as fill it, no more than spreads the block over every CTA
    for (OLBlock& B : k->host_blocks) {
      const int D = 1 << B.k, tpt = D * (D >= kOLSplit ? kOLSplit : D);
      int g = 1;
      while ((g << 1) * tpt <= kOLThreads && (uint64_t)(g << 1) * (uint64_t)grid <= B.ntuples) g <<= 1;
      B.group = g;
    }
    if (nb > 0)
      QS_CUDA(cudaMemcpyAsync(k->blocks, k->host_blocks.data(), sizeof(OLBlock) * nb, cudaMemcpyHostToDevice, st));
    k->grid = grid;
  }
  // scratch: second state buffer | sync | partials
  const uint64_t dim = 1ull << n;
  auto al = [](size_t x) { return (x + 255) / 256 * 256; };
  const size_t o_sync = al(ab * dim), o_part = o_sync + 256, o_out = o_part + al(sizeof(double) * grid);
  QS_TRY(ensure_ws(s, s->ws, o_out + 256));
  char* w = (char*)s->ws.ptr;
  static int* status_of[64] = {nullptr};
  if (!status_of[dev]) QS_TRY(tc_status_address(&status_of[dev]));
  QS_CUDA(cudaMemsetAsync(w + o_sync, 0, sizeof(OLSync), st));
  a.status = status_of[dev];
  a.psi = s->data;
  a.tmp = w;
  a.blocks = k->blocks;
  a.mats = k->mats;
  a.nblocks = nb;
  a.dim = dim;
  a.sync = (OLSync*)(w + o_sync);
  a.partials = (double*)(w + o_part);
  a.out = o ? dev_out : (double*)(w + o_out);
  void* args[] = {&a};
  QS_CUDA(cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(kOLThreads), args, 0, st));
  return QS_OK;
}

}  // extern "C"
