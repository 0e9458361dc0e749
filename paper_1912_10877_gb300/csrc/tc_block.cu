// tc_block.cu -- dense k-qubit blocks (k = 4, 5) on the 5th-generation tensor
// cores (tcgen05, sm_103a), complex64.
//
// The general multi-qubit instruction (Sec. "Performance") applies a 2^k x 2^k
// matrix to every 2^k-tuple of amplitudes.  For a dense block this is a complex
// matrix product; with D = 2^k and W = 2D it becomes one real GEMM per 128
// tuples:
//   A (M = 128 tuples x K = W): row t = [Re x_0 .. Re x_{D-1}, Im x_0 .. Im x_{D-1}]
//   B (N = W outputs x K = W):  the real form of the matrix,
//       Re y_r = sum_c Re U_rc Re x_c - Im U_rc Im x_c
//       Im y_r = sum_c Im U_rc Re x_c + Re U_rc Im x_c
//   D = A B^T (M x N, FP32) in tensor memory.
// FP32 accuracy comes from the 3xTF32 split: v = hi + lo with hi = v with its
// low 13 mantissa bits cleared (exact in TF32) and lo = v - hi (exact in FP32),
// and D = A_hi B_hi + A_hi B_lo + A_lo B_hi; the omitted lo*lo term is below
// 2^-20 of each product.
//
// Per tile of 128 tuples a CTA of 128 threads
//   1. computes the base index of each tuple (thread t: tuple t),
//   2. gathers the 128 x D amplitudes with consecutive threads on consecutive
//      addresses (targets that are the lowest qubits vary fastest, then the
//      tuple), splits them and stores A_hi, A_lo in shared memory,
//   3. has one thread issue the W/8 x 3 tcgen05.mma (kind::tf32, K = 8 each),
//      committed to an mbarrier,
//   4. reads its own row of D back with tcgen05.ld (warp w owns TMEM lanes
//      32w..32w+31) and stages it in shared memory over the consumed A,
//   5. scatters the tile back in the gather's order.
// Operands use the canonical K-major 128-byte-swizzle layout: 8-row atoms of
// 128-byte rows, 16-byte chunk c of row r stored at chunk c ^ (r mod 8), and
// the K extent split into 128-byte column blocks stored one after another.
// Every wait on the mbarrier is bounded in polls and in time; a wait that
// gives up sets a device status word that qs_state_sync reports.
#include <algorithm>
#include <cstring>

#include "common.cuh"

namespace qs {

constexpr int kTcThreads = 128;                     // one thread per tuple row
constexpr int kTcRows = 128;                        // M of the MMA
constexpr uint32_t kTcSpinLimit = 1u << 24;         // mbarrier polls before giving up
constexpr uint64_t kTcTimeLimitNs = 2000000000ull;  // and at most 2 s of wall time

__device__ int g_tc_status;  // 0 = fine; 1 = an MMA completion wait gave up

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// byte offset of fp32 element (row, col) in a K-major SW128 tile of `rows` rows
__host__ __device__ __forceinline__ uint32_t sw128_off(int row, int col, int rows) {
  const int blk = col >> 5;         // 128-byte column block (32 fp32)
  const int c16 = (col & 31) >> 2;  // 16-byte chunk inside the block's row
  return (uint32_t)(blk * rows * 128 + row * 128 + ((c16 ^ (row & 7)) << 4) + ((col & 3) << 2));
}

// shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups
// 1024 bytes apart (stride byte offset), descriptor version 1
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);  // bits 0-13: start address / 16
  d |= (uint64_t)1u << 16;                   // bits 16-29: leading byte offset (unused when swizzled)
  d |= (uint64_t)(1024u >> 4) << 32;         // bits 32-45: stride byte offset / 16
  d |= (uint64_t)1u << 46;                   // bits 46-47: version
  d |= (uint64_t)2u << 61;                   // bits 61-63: 128-byte swizzle
  return d;
}

// instruction descriptor, kind::tf32: D f32, A and B tf32, both K-major, N, M = 128
__host__ __device__ constexpr uint32_t tf32_idesc(int n_dim) {
  return (1u << 4)                            // bits 4-5: D format f32
         | (2u << 7)                          // bits 7-9: A format tf32
         | (2u << 10)                         // bits 10-12: B format tf32
         | ((uint32_t)(n_dim >> 3) << 17)     // bits 17-22: N / 8
         | ((uint32_t)(kTcRows >> 4) << 24);  // bits 24-28: M / 16
}

__device__ __forceinline__ float tf32_hi(float v) { return __uint_as_float(__float_as_uint(v) & 0xFFFFE000u); }

__device__ __forceinline__ void mma_tf32(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void mma_commit(uint32_t mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
               : "memory");
}

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// bounded wait for completion of the mbarrier phase with the given parity
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity) {
  const uint64_t t0 = global_ns();
  for (uint32_t it = 0; it < kTcSpinLimit; ++it) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(mbar), "r"(parity)
        : "memory");
    if (ok) return true;
    if ((it & 255u) == 255u && global_ns() - t0 > kTcTimeLimitNs) return false;
  }
  return false;
}

// 32 lanes x 32 consecutive 32-bit TMEM columns: thread i of the warp gets lane (base lane + i)
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

template <int K>
struct TcArgs {
  float2* psi;
  uint64_t ntuples;          // tuples per register
  uint64_t reg_stride;       // amplitudes per register
  uint64_t total;            // ntuples * registers
  IdxSpec s;                 // tuple base index inside a register (targets and controls fixed)
  int lowbits;               // targets 0..lowbits-1 are register qubits 0..lowbits-1
  uint32_t off[1 << K];      // amplitude offsets of a tuple's members (targets ascending)
  float b[2 << K][2 << K];   // real form of the matrix, [output][input]
};

template <int K>
struct TcSmem {
  static constexpr int D = 1 << K, W = 2 * D;
  static constexpr uint32_t A_BYTES = kTcRows * W * 4;
  static constexpr uint32_t B_BYTES = W * W * 4;
  // offsets from a 1024-aligned base: A_hi, A_lo, B_hi, B_lo, tuple bases,
  // member offsets, mbarrier, TMEM slot
  static constexpr uint32_t A_HI = 0, A_LO = A_BYTES, B_HI = 2 * A_BYTES, B_LO = B_HI + B_BYTES;
  static constexpr uint32_t BASES = B_LO + B_BYTES;
  static constexpr uint32_t OFFS = BASES + kTcRows * 8;
  static constexpr uint32_t MBAR = OFFS + D * 4;
  static constexpr uint32_t TSLOT = MBAR + 8;
  static constexpr uint32_t BYTES = TSLOT + 8 + 1024;  // + alignment slack
  // outputs staged after the MMA has read A: float2 [128][D + 1] over A_hi..A_lo
  static_assert(kTcRows * (D + 1) * 8 <= 2 * A_BYTES, "output staging fits in the A operands");
};

template <int K>
__global__ void __launch_bounds__(kTcThreads) k_block_tc(const __grid_constant__ TcArgs<K> a) {
  using L = TcSmem<K>;
  constexpr int D = L::D, W = L::W;
  extern __shared__ unsigned char sm_raw[];
  unsigned char* sm = (unsigned char*)(((uintptr_t)sm_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* s_base = reinterpret_cast<uint64_t*>(sm + L::BASES);
  uint32_t* s_off = reinterpret_cast<uint32_t*>(sm + L::OFFS);
  float2* s_out = reinterpret_cast<float2*>(sm + L::A_HI);
  uint64_t* mbar = reinterpret_cast<uint64_t*>(sm + L::MBAR);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + L::TSLOT);
  const int tid = threadIdx.x, warp = tid >> 5;
  const int lb = a.lowbits;
  const uint32_t lowmask = (1u << lb) - 1u;

  // the matrix (hi / lo) and the member offsets once per CTA
  if (tid < D) s_off[tid] = a.off[tid];
  for (int e = tid; e < W * W; e += kTcThreads) {
    const int n = e / W, kk = e % W;
    const float v = a.b[n][kk], h = tf32_hi(v);
    *reinterpret_cast<float*>(sm + L::B_HI + sw128_off(n, kk, W)) = h;
    *reinterpret_cast<float*>(sm + L::B_LO + sw128_off(n, kk, W)) = v - h;
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(mbar)));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                 "r"((uint32_t)W));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tslot;
  const uint32_t mb = smem_u32(mbar);
  const uint32_t a_hi = smem_u32(sm + L::A_HI), a_lo = smem_u32(sm + L::A_LO);
  const uint32_t b_hi = smem_u32(sm + L::B_HI), b_lo = smem_u32(sm + L::B_LO);
  uint32_t parity = 0;
  bool failed = false;

  for (uint64_t t0 = (uint64_t)blockIdx.x * kTcRows; t0 < a.total; t0 += (uint64_t)gridDim.x * kTcRows) {
    {  // 1. tuple bases
      const uint64_t t = t0 + tid;
      uint64_t b = 0;
      if (t < a.total) {
        const uint64_t r = t / a.ntuples, j = t - r * a.ntuples;
        b = r * a.reg_stride + deposit(j, a.s);
      }
      s_base[tid] = b;
    }
    __syncthreads();
    const int rows = a.total - t0 < (uint64_t)kTcRows ? (int)(a.total - t0) : kTcRows;
    // 2. gather: element e -> m_lo = e mod 2^lb, t = (e >> lb) mod 128, m_hi = e >> (lb + 7)
    {
      float2 v[D];
#pragma unroll
      for (int i = 0; i < D; ++i) {
        const uint32_t e = (uint32_t)tid + (uint32_t)i * kTcThreads;
        const int t = (int)((e >> lb) & (kTcRows - 1));
        const uint32_t m = (e & lowmask) | ((e >> (lb + 7)) << lb);
        v[i] = t < rows ? a.psi[s_base[t] + s_off[m]] : make_float2(0.f, 0.f);
      }
#pragma unroll
      for (int i = 0; i < D; ++i) {
        const uint32_t e = (uint32_t)tid + (uint32_t)i * kTcThreads;
        const int t = (int)((e >> lb) & (kTcRows - 1));
        const int m = (int)((e & lowmask) | ((e >> (lb + 7)) << lb));
        const float hr = tf32_hi(v[i].x), hm = tf32_hi(v[i].y);
        *reinterpret_cast<float*>(sm + L::A_HI + sw128_off(t, m, kTcRows)) = hr;
        *reinterpret_cast<float*>(sm + L::A_LO + sw128_off(t, m, kTcRows)) = v[i].x - hr;
        *reinterpret_cast<float*>(sm + L::A_HI + sw128_off(t, D + m, kTcRows)) = hm;
        *reinterpret_cast<float*>(sm + L::A_LO + sw128_off(t, D + m, kTcRows)) = v[i].y - hm;
      }
    }
    // generic-proxy stores -> visible to the tensor core (async proxy)
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    // 3. one thread issues the MMA chain
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      constexpr uint32_t idesc = tf32_idesc(W);
#pragma unroll
      for (int ks = 0; ks < W / 8; ++ks) {
        const uint32_t koff = (uint32_t)(ks & 3) * 32u;  // 8 tf32 = 32 bytes inside a 128-byte block
        const uint32_t ablk = (uint32_t)(ks >> 2) * (uint32_t)(kTcRows * 128);
        const uint32_t bblk = (uint32_t)(ks >> 2) * (uint32_t)(W * 128);
        const uint64_t dah = sw128_desc(a_hi + ablk + koff), dal = sw128_desc(a_lo + ablk + koff);
        const uint64_t dbh = sw128_desc(b_hi + bblk + koff), dbl = sw128_desc(b_lo + bblk + koff);
        mma_tf32(tmem, dah, dbh, idesc, ks > 0 ? 1u : 0u);
        mma_tf32(tmem, dah, dbl, idesc, 1u);
        mma_tf32(tmem, dal, dbh, idesc, 1u);
      }
      mma_commit(mb);
    }
    // 4. bounded wait, then this thread's row of D
    const bool ok = mbar_wait(mb, parity);
    parity ^= 1u;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (__syncthreads_or(ok ? 0 : 1)) {
      failed = true;
      break;
    }
    {
      float y[W];
#pragma unroll
      for (int c = 0; c < W; c += 32) tmem_ld32(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)c, y + c);
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      // the MMA has finished reading A: stage the outputs over it, row stride D + 1 (bank spread)
#pragma unroll
      for (int m = 0; m < D; ++m) s_out[tid * (D + 1) + m] = make_float2(y[m], y[D + m]);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    // 5. scatter in the gather's order
#pragma unroll 4
    for (int i = 0; i < D; ++i) {
      const uint32_t e = (uint32_t)tid + (uint32_t)i * kTcThreads;
      const int t = (int)((e >> lb) & (kTcRows - 1));
      const uint32_t m = (e & lowmask) | ((e >> (lb + 7)) << lb);
      if (t < rows) a.psi[s_base[t] + s_off[m]] = s_out[t * (D + 1) + m];
    }
    __syncthreads();  // A, the staged outputs and the tuple bases are free for the next tile
  }
  if (failed) {
    if (tid == 0) atomicExch(&g_tc_status, 1);
    // one more bounded wait for the MMA still in flight before its TMEM is freed
    mbar_wait(mb, parity ^ 1u);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  }
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)W));
}

template <int K>
static int launch_tc_t(float2* psi, int n, int nreg, const Plan& p, cudaStream_t st) {
  using L = TcSmem<K>;
  constexpr int D = L::D;
  TcArgs<K> a;
  memset(&a, 0, sizeof(a));
  // targets in ascending qubit order; the matrix's row and column bits follow
  int order[K];
  for (int j = 0; j < K; ++j) order[j] = j;
  std::sort(order, order + K, [&](int x, int y) { return p.locs[x] < p.locs[y]; });
  auto orig = [&](int ms) {  // matrix index (bit j <-> p.locs[j]) of sorted-bit index ms
    int m = 0;
    for (int j = 0; j < K; ++j)
      if ((ms >> j) & 1) m |= 1 << order[j];
    return m;
  };
  uint64_t locmask = 0;
  for (int j = 0; j < K; ++j) locmask |= 1ull << p.locs[j];
  a.lowbits = 0;
  while (a.lowbits < K && p.locs[order[a.lowbits]] == a.lowbits) ++a.lowbits;
  for (int m = 0; m < D; ++m) {
    uint64_t o = 0;
    for (int j = 0; j < K; ++j)
      if ((m >> j) & 1) o |= 1ull << p.locs[order[j]];
    if (o >> 32) return fail(QS_EUNSUPPORTED, "tensor-core blocks take targets below qubit 32");
    a.off[m] = (uint32_t)o;
  }
  for (int r = 0; r < D; ++r)
    for (int c = 0; c < D; ++c) {
      const cd u = p.U[orig(r) * D + orig(c)];
      const float ur = (float)u.real(), ui = (float)u.imag();
      a.b[r][c] = ur;
      a.b[r][D + c] = -ui;
      a.b[D + r][c] = ui;
      a.b[D + r][D + c] = ur;
    }
  QS_TRY(make_idx(n, locmask | p.ctrl_mask, p.ctrl_vals, &a.s));
  a.psi = psi;
  a.ntuples = 1ull << a.s.item_log2;
  a.reg_stride = 1ull << n;
  a.total = a.ntuples * (uint64_t)nreg;
  if (a.total == 0) return QS_OK;
  const size_t smem = L::BYTES;
  int dev = 0, sms = 0, per_sm = 0;
  QS_CUDA(cudaGetDevice(&dev));
  QS_CUDA(cudaFuncSetAttribute(k_block_tc<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  QS_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  QS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_block_tc<K>, kTcThreads, smem));
  if (per_sm < 1) return fail(QS_EDEVICE, "tensor-core block kernel does not fit on an SM");
  // every resident CTA holds W = 2D TMEM columns; an SM has 512
  per_sm = std::min(per_sm, 512 / (2 * D));
  const uint64_t tiles = (a.total + kTcRows - 1) / kTcRows;
  const unsigned grid = (unsigned)std::min<uint64_t>(tiles, (uint64_t)sms * per_sm);
  k_block_tc<K><<<grid, kTcThreads, smem, st>>>(a);
  QS_LAUNCHED();
  return QS_OK;
}

static int g_tc_enabled = 1;

void set_tensor_cores(int on) { g_tc_enabled = on ? 1 : 0; }
int tensor_cores_enabled() { return g_tc_enabled; }

bool use_block_tc(int dtype, const Plan& p) {
  return g_tc_enabled && dtype == QS_C64 && p.op == OP_DENSEK && (p.k == 4 || p.k == 5);
}

int launch_block_tc(float2* psi, int n, int nreg, const Plan& p, cudaStream_t st) {
  if (p.k == 4) return launch_tc_t<4>(psi, n, nreg, p, st);
  if (p.k == 5) return launch_tc_t<5>(psi, n, nreg, p, st);
  return fail(QS_EUNSUPPORTED, "tensor-core blocks take 4 or 5 targets");
}

// reads and clears the device status word (synchronous)
int tc_status_take() {
  int e = 0;
  QS_CUDA(cudaMemcpyFromSymbol(&e, g_tc_status, sizeof(int)));
  if (e) {
    const int z = 0;
    QS_CUDA(cudaMemcpyToSymbol(g_tc_status, &z, sizeof(int)));
    return fail(QS_ETIMEDOUT, "a tensor-core MMA completion wait gave up");
  }
  return QS_OK;
}

}  // namespace qs
