// tc_block.cu -- dense k-qubit blocks (k = 4, 5) on the 5th-generation tensor
// cores (tcgen05, sm_103a), complex64.
//
// The general multi-qubit instruction (Sec. "Performance") applies a 2^k x 2^k
// matrix U to every 2^k-tuple of amplitudes.  For a dense block this is a
// complex matrix product; with D = 2^k and W = 2D it becomes one real GEMM per
// 128 tuples, with real and imaginary parts interleaved as they are in memory:
//   A (M = 128 tuples x K = W): row t = [Re x_0, Im x_0, Re x_1, Im x_1, ...]
//   B (N = W x K = W), the real form of U:
//       B[2r][2c] = Re U_rc   B[2r][2c+1] = -Im U_rc
//       B[2r+1][2c] = Im U_rc B[2r+1][2c+1] = Re U_rc
//   C = A B^T (M x N, FP32) in tensor memory: row t = [Re y_0, Im y_0, ...].
// FP32 accuracy comes from the 3xTF32 split: v = hi + lo with hi = v with its
// low 13 mantissa bits cleared (exact in TF32) and lo = v - hi (exact in FP32),
// and C = A_hi B_hi + A_hi B_lo + A_lo B_hi; the omitted lo*lo term is below
// 2^-20 of each product.
//
// One persistent CTA per SM, warp-specialised, tiles of 128 tuples:
//   warps 0-15  load a tile with 16-byte accesses (the loads of the tile
//               two ahead are in flight while the current one is split into
//               A_hi / A_lo in one of two shared-memory stages),
//   warp 24     issues the W/8 x 3 tcgen05.mma (kind::tf32, K = 8 each) into
//               one of two TMEM accumulators and commits them to mbarriers,
//   warps 16-23 read the accumulator rows back with one tcgen05.ld of 32
//               columns each (warp w owns TMEM lanes 32 (w mod 4) .. and
//               columns 32 ((w - 16) / 4) ..) and store them to global memory
//               (through a shared-memory staging tile where a row is a run of
//               adjacent amplitudes, so that the stores stay coalesced).
// Per-role timestamps showed a tile costing about as long as four epilogue
// warps took to drain it (two dependent TMEM loads, then staging and stores)
// while the MMA warp waited for the accumulator; eight warps halve that.
// Operands use the canonical K-major 128-byte-swizzle layout: 8-row atoms of
// 128-byte rows, 16-byte chunk c of row r stored at chunk c ^ (r mod 8), and
// the K extent split into 128-byte column blocks stored one after another.
// Every mbarrier wait is bounded in polls and in time; a wait that gives up
// raises a CTA-wide abort flag, sets a device status word that qs_state_sync
// reports, and every role leaves its loop; the MMA warp waits (bounded) for
// its last commit before the TMEM is freed.
#include <algorithm>
#include <cstring>
#include <type_traits>

#include <cuda.h>

#include "common.cuh"

namespace qs {

constexpr int kTcRows = 128;                        // M of the MMA: tuples per tile
constexpr int kTcLoadWarps = 16, kTcEpiWarps = 4;
constexpr int kTcLoaders = kTcLoadWarps * 32;       // 512
constexpr int kTcEpiWarp0 = kTcLoadWarps;           // warps 16..19 (TMEM lane quarters 0..3)
constexpr int kTcMmaWarp = kTcLoadWarps + kTcEpiWarps;  // warp 20
constexpr int kTcThreads = (kTcMmaWarp + 1) * 32;   // 672
// k_block_tc drains its accumulators with eight epilogue warps: warp 16 + e
// reads TMEM lane quarter e mod 4 (the quarter a warp may access is its warp
// index mod 4) and accumulator columns 32 (e / 4) .. 32 (e / 4) + 31
constexpr int kBkEpiWarps = 8;
constexpr int kBkEpiThreads = kBkEpiWarps * 32;      // 256
constexpr int kBkMmaWarp = kTcLoadWarps + kBkEpiWarps;  // warp 24
constexpr int kBkThreads = (kBkMmaWarp + 1) * 32;   // 800
constexpr uint32_t kTcSpinLimit = 1u << 20;         // mbarrier polls before giving up
constexpr uint64_t kTcTimeLimitNs = 2000000000ull;  // and at most 2 s of wall time

// how a loader thread's 16-byte (or 8-byte) unit maps onto the tile
enum { TC_PAIR_MEMBERS = 0,  // target qubit 0: members (2q, 2q+1) of one tuple are adjacent
       TC_PAIR_TUPLES = 1,   // qubit 0 free: tuples (2p, 2p+1) of one member are adjacent
       TC_SCALAR = 2 };      // qubit 0 is a control (or one tuple per register): 8-byte units

__device__ int g_tc_status;  // 0 = fine; 1 = an MMA pipeline wait gave up

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

// K-major 32-byte-swizzle layout for operands read 8 tf32 (32 bytes) per row
// per MMA: K step ks of a `rows`-row operand is a block of rows x 32 bytes at
// ks x rows x 32, 8-row atoms 256 bytes apart, 16-byte chunk index XOR row bit 2
// (with the 128-byte swizzle a K = 8 MMA reads 32 of every 128-byte row, and
// MMAs with both operands in shared memory ran at half the rate of the block
// kernel's, whose A operand is in tensor memory)
__host__ __device__ __forceinline__ uint32_t sw32_off(int row, int k, int rows) {
  const int ks = k >> 3, kk = k & 7;
  return (uint32_t)(ks * rows * 32 + row * 32 + ((((kk >> 2) & 1) ^ ((row >> 2) & 1)) << 4) + ((kk & 3) << 2));
}
__device__ __forceinline__ uint64_t sw32_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);  // start address / 16
  d |= (uint64_t)1u << 16;                   // leading byte offset (unused when swizzled)
  d |= (uint64_t)(256u >> 4) << 32;          // stride byte offset: 8-row atoms of 8 x 32 bytes
  d |= (uint64_t)1u << 46;                   // version
  d |= (uint64_t)6u << 61;                   // 32-byte swizzle
  return d;
}

// instruction descriptor, kind::tf32: D f32, A and B tf32, both K-major, N, M (128 by default)
__host__ __device__ constexpr uint32_t tf32_idesc(int n_dim, int m_dim = kTcRows) {
  return (1u << 4)                            // bits 4-5: D format f32
         | (2u << 7)                          // bits 7-9: A format tf32
         | (2u << 10)                         // bits 10-12: B format tf32
         | ((uint32_t)(n_dim >> 3) << 17)     // bits 17-22: N / 8
         | ((uint32_t)(m_dim >> 4) << 24);    // bits 24-28: M / 16
}

// v rounded to the nearest TF32 value (10 stored mantissa bits, ties away from
// zero): exactly representable, so the tensor core reads it unchanged
__device__ __forceinline__ float tf32_hi(float v) { return __uint_as_float((__float_as_uint(v) + 0x1000u) & 0xFFFFE000u); }
// the correction v - hi (exact in FP32), itself rounded to TF32: hi + lo = v to
// 2^-24 relative, unbiased (a lo left in FP32 would be truncated by the tensor
// core, a bias of up to 2^-22 that accumulates over blocks)
__device__ __forceinline__ float tf32_lo(float v, float h) { return tf32_hi(v - h); }

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

__device__ __forceinline__ void mbar_init(uint32_t mbar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(mbar), "r"(count));
}

__device__ __forceinline__ void mbar_arrive(uint32_t mbar) {
  asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}\n" ::"r"(mbar) : "memory");
}

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// bounded wait for completion of the mbarrier phase with the given parity;
// gives up (and raises *abort) after limit_ns of wall time or kTcSpinLimit
// polls, or when another role has raised *abort.  Each try_wait may suspend
// the thread for up to 20 us while the phase is incomplete, so polls are few
// and the poll cap alone bounds the wait (2^20 x 20 us = 21 s).
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity, volatile int* abort,
                                          uint64_t limit_ns = kTcTimeLimitNs) {
  uint64_t t0 = 0;
  for (uint32_t it = 0; it < kTcSpinLimit; ++it) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(mbar), "r"(parity), "r"(20000u)
        : "memory");
    if (ok) return true;
    if (*abort) return false;
    const uint64_t now = global_ns();
    if (it == 0) t0 = now;
    else if (now - t0 > limit_ns) break;
  }
  *abort = 1;
  return false;
}

// named barrier over `n` threads, OR-reducing a predicate
__device__ __forceinline__ bool bar_or(int id, int n, bool p) {
  uint32_t r;
  asm volatile(
      "{\n\t.reg .pred pi, po;\n\tsetp.ne.u32 pi, %1, 0;\n\t"
      "bar.red.or.pred po, %2, %3, pi;\n\tselp.u32 %0, 1, 0, po;\n\t}\n"
      : "=r"(r)
      : "r"((uint32_t)p), "r"(id), "r"(n)
      : "memory");
  return r != 0;
}
__device__ __forceinline__ void bar_sync(int id, int n) { asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory"); }

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
  uint64_t total;            // tuples over all registers
  uint64_t reg_stride;       // amplitudes per register
  int lg;                    // log2(tuples per register)
  int lowbits;               // targets 0..lowbits-1 are register qubits 0..lowbits-1
  IdxSpec s;                 // tuple base index inside a register (targets and controls fixed)
  uint32_t off[1 << K];      // amplitude offsets of a tuple's members (targets ascending)
  float b[2 << K][2 << K];   // real form of the matrix, [output column][input column]
};

template <int K>
struct TcSmem {
  static constexpr int D = 1 << K, W = 2 * D;
  static constexpr uint32_t A_BYTES = kTcRows * W * 4;
  static constexpr uint32_t B_BYTES = W * W * 4;
  // offsets from a 1024-aligned base
  static constexpr uint32_t A0 = 0;                        // stage s: hi at A0 + 2s A_BYTES, lo after it
  static constexpr uint32_t B_HI = 4 * A_BYTES, B_LO = B_HI + B_BYTES;
  static constexpr uint32_t ROWOFF = B_LO + B_BYTES;       // P[t]: row t's index relative to its tile
  static constexpr uint32_t DTAB = ROWOFF + kTcRows * 8;   // deposit of tuple-index byte c (bits 7+8c..)
  static constexpr uint32_t OFFS = DTAB + 4 * 256 * 8;
  static constexpr uint32_t MBAR = OFFS + D * 4;           // full[2], empty[2], tfull[2], tempty[2], fin
  static constexpr uint32_t FLAGS = MBAR + 9 * 8;          // TMEM address, abort flag
  // epilogue staging when a row holds runs of >= 4 adjacent amplitudes:
  // float2 [128][D + 2] (the row stride is an odd number of 16-byte chunks,
  // so rows written by consecutive threads fall in distinct banks)
  static constexpr int SROW = D + 2;
  static constexpr uint32_t STAGE = (FLAGS + 16 + 15) & ~15u;
  static constexpr uint32_t BYTES = STAGE + kTcRows * SROW * 8 + 1024;  // + alignment slack
  __host__ __device__ static constexpr uint32_t a_hi(int s) { return A0 + (uint32_t)s * 2 * A_BYTES; }
};

// Amplitude index of tuple t0 + t (t0 a multiple of 128, t < 128) is
// tile_base(t0) + P[t]: the register and tuple bits of t0 and of t are disjoint
// (tuples per register and 128 are powers of two), and deposit is a bit scatter.
__device__ __forceinline__ uint64_t deposit_nb(uint64_t j, const IdxSpec& s) { return deposit(j, s) & ~s.set_bits; }

// deposit of the tuple-index bits 7.. of t0 through per-byte tables
// (dtab[c][v] = deposit of v << (7 + 8c)); indices up to 2^39 tuples
template <int K>
__device__ __forceinline__ uint64_t tile_base(uint64_t t0, const TcArgs<K>& a, const uint64_t* dtab) {
  uint64_t b = (t0 >> a.lg) * a.reg_stride + a.s.set_bits;
  if (a.lg > 7) {
    const uint64_t j = (t0 & ((1ull << a.lg) - 1ull)) >> 7;
#pragma unroll
    for (int c = 0; c < 4; ++c) b |= dtab[c * 256 + (int)((j >> (8 * c)) & 255u)];
  }
  return b;
}

template <int K>
__device__ __forceinline__ uint64_t row_offset(int t, const TcArgs<K>& a) {
  if (a.lg >= 7) return deposit_nb((uint64_t)t, a.s);
  return (uint64_t)(t >> a.lg) * a.reg_stride + deposit_nb((uint64_t)t & ((1ull << a.lg) - 1ull), a.s);
}

template <int K, int MODE>
__global__ void __launch_bounds__(kBkThreads, 1) k_block_tc(const __grid_constant__ TcArgs<K> a) {
  using L = TcSmem<K>;
  constexpr int D = L::D, W = L::W;
  constexpr uint32_t A_BYTES = L::A_BYTES;
  // units (16 bytes: two amplitudes; 8 bytes in TC_SCALAR) per tile and per loader thread
  constexpr int NU = MODE == TC_SCALAR ? kTcRows * D : kTcRows * D / 2;
  constexpr int UT = NU / kTcLoaders;
  static_assert(UT * kTcLoaders == NU && UT <= 8, "tile splits evenly over the loaders");
  using VT = typename std::conditional<MODE == TC_SCALAR, float2, float4>::type;

  extern __shared__ unsigned char sm_raw[];
  unsigned char* sm = (unsigned char*)(((uintptr_t)sm_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* s_P = reinterpret_cast<uint64_t*>(sm + L::ROWOFF);
  uint32_t* s_off = reinterpret_cast<uint32_t*>(sm + L::OFFS);
  const uint32_t mb0 = smem_u32(sm + L::MBAR);
  auto full = [&](int s) { return mb0 + 8u * (uint32_t)s; };
  auto empty = [&](int s) { return mb0 + 16u + 8u * (uint32_t)s; };
  auto tfull = [&](int s) { return mb0 + 32u + 8u * (uint32_t)s; };
  auto tempty = [&](int s) { return mb0 + 48u + 8u * (uint32_t)s; };
  const uint32_t fin = mb0 + 64u;
  uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + L::FLAGS);
  volatile int* abort = reinterpret_cast<volatile int*>(sm + L::FLAGS + 4);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  // ---- setup: the matrix (hi / lo), member and row offsets, barriers, TMEM
  for (int e = tid; e < W * W; e += kBkThreads) {
    const int n = e / W, kk = e % W;
    const float v = a.b[n][kk], h = tf32_hi(v);
    *reinterpret_cast<float*>(sm + L::B_HI + sw128_off(n, kk, W)) = h;
    *reinterpret_cast<float*>(sm + L::B_LO + sw128_off(n, kk, W)) = tf32_lo(v, h);
  }
  if (tid < D) s_off[tid] = a.off[tid];
  if (tid < kTcRows) s_P[tid] = row_offset(tid, a);
  uint64_t* s_dtab = reinterpret_cast<uint64_t*>(sm + L::DTAB);
  for (int e = tid; e < 4 * 256; e += kBkThreads) {
    const int c = e >> 8, sh = 7 + 8 * c;
    const uint64_t v = (uint64_t)(e & 255) << sh;
    s_dtab[e] = (sh < a.lg) ? deposit_nb(v & ((1ull << a.lg) - 1ull), a.s) : 0;
  }
  if (tid == 0) {
    for (int s = 0; s < 2; ++s) {
      mbar_init(full(s), kTcLoaders);
      mbar_init(empty(s), 1);
      mbar_init(tfull(s), 1);
      mbar_init(tempty(s), (W / 32) * 4 * 32);
    }
    mbar_init(fin, 1);
    *abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == kBkMmaWarp) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                 "r"((uint32_t)(2 * W)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  // B written by the generic proxy is read by the tensor core
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tslot;
  const uint64_t stride_tiles = (uint64_t)gridDim.x;
  auto tile_row0 = [&](int i) { return ((uint64_t)blockIdx.x + (uint64_t)i * stride_tiles) * kTcRows; };
  auto tile_rows = [&](uint64_t t0) {
    return a.total - t0 < (uint64_t)kTcRows ? (int)(a.total - t0) : kTcRows;
  };

  if (warp < kTcLoadWarps) {
    // ================================================================ loaders
    // Every loader thread owns the same UT units of every tile: their global
    // offsets (relative to the tile base) and shared-memory slots are computed
    // once.  Threads run independently: the stage mbarriers are the only sync.
    const int lt = tid;
    const int lb = a.lowbits;
    uint64_t goff[UT];
    uint32_t soff[UT];
    uint32_t trows = 0;  // the units' rows, 8 bits each (UT <= 4)
    int tmax = 0;
#pragma unroll
    for (int k = 0; k < UT; ++k) {
      const int u = lt + k * kTcLoaders;
      int t, m;
      if (MODE == TC_PAIR_MEMBERS) {
        const int hb = lb - 1;
        t = (u >> hb) & (kTcRows - 1);
        m = 2 * ((u & ((1 << hb) - 1)) | ((u >> (hb + 7)) << hb));
      } else if (MODE == TC_PAIR_TUPLES) {
        t = 2 * (u & (kTcRows / 2 - 1));
        m = u >> 6;
      } else {
        t = u & (kTcRows - 1);
        m = u >> 7;
      }
      goff[k] = s_P[t] + s_off[m];
      soff[k] = sw128_off(t, 2 * m, kTcRows);  // PAIR_TUPLES: row t + 1 is at sw128_off(t + 1, 2m)
      if (UT <= 4) trows |= (uint32_t)t << (8 * k);
      tmax = max(tmax, MODE == TC_PAIR_TUPLES ? t + 1 : t);
    }
    VT v0[UT], v1[UT], v2[UT];
    auto load = [&](uint64_t t0, VT* v) {
      const uint64_t tb = tile_base(t0, a, s_dtab);
      const int rows = tile_rows(t0);
      if (tmax < rows) {
#pragma unroll
        for (int k = 0; k < UT; ++k) v[k] = *reinterpret_cast<const VT*>(a.psi + tb + goff[k]);
      } else {  // the last, partial tile
#pragma unroll
        for (int k = 0; k < UT; ++k) {
          // UT > 4 only in TC_SCALAR, where every unit of a thread is in row lt mod 128
          const int t = UT <= 4 ? (int)((trows >> (8 * k)) & 255u) : (lt & (kTcRows - 1));
          v[k] = t < rows ? *reinterpret_cast<const VT*>(a.psi + tb + goff[k]) : VT{};
        }
      }
    };
    auto split_store = [&](const VT* v, int s) {
      unsigned char* ah = sm + L::a_hi(s);
      unsigned char* al = ah + A_BYTES;
#pragma unroll
      for (int k = 0; k < UT; ++k) {
        if (MODE == TC_PAIR_MEMBERS) {
          const float4 x = *reinterpret_cast<const float4*>(&v[k]);
          const float4 h = make_float4(tf32_hi(x.x), tf32_hi(x.y), tf32_hi(x.z), tf32_hi(x.w));
          *reinterpret_cast<float4*>(ah + soff[k]) = h;  // columns 2m..2m+3: one 16-byte chunk
          *reinterpret_cast<float4*>(al + soff[k]) =
              make_float4(tf32_lo(x.x, h.x), tf32_lo(x.y, h.y), tf32_lo(x.z, h.z), tf32_lo(x.w, h.w));
        } else if (MODE == TC_PAIR_TUPLES) {
          const float4 x = *reinterpret_cast<const float4*>(&v[k]);
          const float2 h0 = make_float2(tf32_hi(x.x), tf32_hi(x.y)), h1 = make_float2(tf32_hi(x.z), tf32_hi(x.w));
          // row t + 1 of the same column: next 128-byte row, chunk index ^ 1 when t is even
          const uint32_t o0 = soff[k], o1 = (o0 + 128u) ^ 16u;
          *reinterpret_cast<float2*>(ah + o0) = h0;
          *reinterpret_cast<float2*>(al + o0) = make_float2(tf32_lo(x.x, h0.x), tf32_lo(x.y, h0.y));
          *reinterpret_cast<float2*>(ah + o1) = h1;
          *reinterpret_cast<float2*>(al + o1) = make_float2(tf32_lo(x.z, h1.x), tf32_lo(x.w, h1.y));
        } else {
          const float2 x = *reinterpret_cast<const float2*>(&v[k]);
          const float2 h = make_float2(tf32_hi(x.x), tf32_hi(x.y));
          *reinterpret_cast<float2*>(ah + soff[k]) = h;
          *reinterpret_cast<float2*>(al + soff[k]) = make_float2(tf32_lo(x.x, h.x), tf32_lo(x.y, h.y));
        }
      }
    };
    // tile i is split from one of three register buffers while the loads of
    // tile i + 2 are in flight in another (the loop body is unrolled over the
    // rotation, so no register copies wait on loads)
    auto step = [&](int i, const VT* vc, VT* vp) -> bool {
      if (tile_row0(i) >= a.total) return false;
      const int s = i & 1;
      const uint64_t tn = tile_row0(i + 2);
      if (tn < a.total) load(tn, vp);
      // the stage is free once the MMAs that read it two tiles ago have completed
      if (!mbar_wait(empty(s), ((i >> 1) & 1) ^ 1, abort)) return false;
      split_store(vc, s);
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      mbar_arrive(full(s));
      return true;
    };
    if (tile_row0(0) < a.total) load(tile_row0(0), v0);
    if (tile_row0(1) < a.total) load(tile_row0(1), v1);
    for (int i = 0;; i += 3) {
      if (!step(i, v0, v2)) break;
      if (!step(i + 1, v1, v0)) break;
      if (!step(i + 2, v2, v1)) break;
    }
  } else if (warp < kBkMmaWarp) {
    // ================================================================ epilogue
    const int e = warp - kTcEpiWarp0;           // 0..7
    const int q = warp & 3;                     // TMEM lane quarter
    const int c = 32 * (e >> 2);                // first accumulator column of this warp
    const bool reads = c < W;                   // 4-qubit blocks: warps 20..23 only store
    const int t = q * 32 + lane;                // this thread's row of every tile
    const int et = e * 32 + lane;               // 0..255
    const uint64_t myP = s_P[t];
    const bool staged = MODE == TC_PAIR_MEMBERS && a.lowbits >= 2;
    float2* stage = reinterpret_cast<float2*>(sm + L::STAGE);
    for (int i = 0; tile_row0(i) < a.total; ++i) {
      const int s = i & 1;
      const uint64_t t0 = tile_row0(i);
      const int rows = tile_rows(t0);
      const bool valid = t < rows;
      const uint64_t tb = tile_base(t0, a, s_dtab);
      const uint64_t base = tb + myP;
      // the eight epilogue warps agree on giving up (they share named barrier 2)
      if (bar_or(2, kBkEpiThreads, !mbar_wait(tfull(s), (i >> 1) & 1, abort))) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      if (reads) {
        // 32 columns (16 amplitudes); the accumulator half is released right after the load
        float y[32];
        tmem_ld32(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(s * W + c), y);
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        mbar_arrive(tempty(s));
        const int m0 = c / 2;
        if (staged) {
          // stage the row; it leaves in coalesced runs below
#pragma unroll
          for (int m = 0; m < 16; m += 2)
            *reinterpret_cast<float4*>(stage + t * L::SROW + m0 + m) =
                make_float4(y[2 * m], y[2 * m + 1], y[2 * m + 2], y[2 * m + 3]);
        } else if (valid) {
          // consecutive rows hold adjacent amplitudes (or pairs): coalesced stores
          if (MODE == TC_PAIR_MEMBERS) {
#pragma unroll
            for (int m = 0; m < 16; m += 2)
              *reinterpret_cast<float4*>(a.psi + base + s_off[m0 + m]) =
                  make_float4(y[2 * m], y[2 * m + 1], y[2 * m + 2], y[2 * m + 3]);
          } else {
#pragma unroll
            for (int m = 0; m < 16; ++m) a.psi[base + s_off[m0 + m]] = make_float2(y[2 * m], y[2 * m + 1]);
          }
        }
      }
      if (staged) {
        bar_sync(2, kBkEpiThreads);
        const int hb = a.lowbits - 1;
        // 64 D 16-byte units per tile, D / 4 per thread
#pragma unroll 4
        for (int k = 0; k < D / 4; ++k) {
          const int u = et + k * kBkEpiThreads;
          const int qq = (u & ((1 << hb) - 1)) | ((u >> (hb + 7)) << hb);
          const int tt = (u >> hb) & (kTcRows - 1);
          if (tt < rows)
            *reinterpret_cast<float4*>(a.psi + tb + s_P[tt] + s_off[2 * qq]) =
                *reinterpret_cast<const float4*>(stage + tt * L::SROW + 2 * qq);
        }
        bar_sync(2, kBkEpiThreads);  // the staging buffer is free for the next tile
      }
    }
    __syncwarp();
  } else {
    // ================================================================ MMA issue
    if (lane == 0) {
      constexpr uint32_t idesc = tf32_idesc(W);
      const uint32_t b_hi = smem_u32(sm + L::B_HI), b_lo = smem_u32(sm + L::B_LO);
      bool issued = false;
      for (int i = 0; tile_row0(i) < a.total; ++i) {
        const int s = i & 1;
        const uint32_t ph = (uint32_t)(i >> 1) & 1u;
        if (!mbar_wait(full(s), ph, abort)) break;
        if (!mbar_wait(tempty(s), ph ^ 1u, abort)) break;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t a_hi = smem_u32(sm + L::a_hi(s)), a_lo = a_hi + A_BYTES;
        const uint32_t d = tmem + (uint32_t)(s * W);
        // the small hi x lo and lo x hi terms first, then hi x hi: the MMA truncates
        // its FP32 sum toward zero, so the large terms should pass through the
        // accumulator as few times as possible (W / 8 instead of 3 W / 8)
#pragma unroll
        for (int pass = 0; pass < 2; ++pass)
#pragma unroll
          for (int ks = 0; ks < W / 8; ++ks) {
            const uint32_t koff = (uint32_t)(ks & 3) * 32u;  // 8 tf32 = 32 bytes inside a 128-byte block
            const uint32_t ablk = (uint32_t)(ks >> 2) * (uint32_t)(kTcRows * 128);
            const uint32_t bblk = (uint32_t)(ks >> 2) * (uint32_t)(W * 128);
            const uint64_t dah = sw128_desc(a_hi + ablk + koff), dal = sw128_desc(a_lo + ablk + koff);
            const uint64_t dbh = sw128_desc(b_hi + bblk + koff), dbl = sw128_desc(b_lo + bblk + koff);
            if (pass == 0) {
              mma_tf32(d, dah, dbl, idesc, ks > 0 ? 1u : 0u);
              mma_tf32(d, dal, dbh, idesc, 1u);
            } else {
              mma_tf32(d, dah, dbh, idesc, 1u);
            }
          }
        mma_commit(empty(s));
        mma_commit(tfull(s));
        issued = true;
      }
      // every MMA issued above has completed once this commit arrives
      if (issued) {
        mma_commit(fin);
        volatile int never = 0;
        mbar_wait(fin, 0, &never);
      }
    }
    __syncwarp();
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (tid == 0 && *abort) atomicExch(&g_tc_status, 1);
  if (warp == kBkMmaWarp)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)(2 * W)));
}

template <int K, int MODE>
static int launch_tc_mode(const TcArgs<K>& a, cudaStream_t st) {
  using L = TcSmem<K>;
  const size_t smem = L::BYTES;
  int dev = 0, sms = 0;
  QS_CUDA(cudaGetDevice(&dev));
  QS_CUDA(cudaFuncSetAttribute(k_block_tc<K, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  QS_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const uint64_t tiles = (a.total + kTcRows - 1) / kTcRows;
  const unsigned grid = (unsigned)std::min<uint64_t>(tiles, (uint64_t)sms);
  k_block_tc<K, MODE><<<grid, kBkThreads, smem, st>>>(a);
  QS_LAUNCHED();
  return QS_OK;
}

// ------------------------------------------------------------------ TMA-fed blocks on consecutive targets
//
// Dense blocks on consecutive targets q .. q+K-1 without controls (every block
// the planner forms from layered and brickwork circuits).  One producer thread
// brings each 128-tuple tile into a ring of shared-memory stages with one TMA
// tensor copy (completion counted in bytes on the stage's mbarrier), so the
// ring depth, not the registers of loader threads, sets the bytes in flight.
// Sixteen converter warps read a tile's FP32 values, split them (hi = v with
// the low 13 mantissa bits cleared, lo = v - hi) and write both into tensor
// memory with tcgen05.st, where the MMAs read the A operand; shared memory
// holds only the ring, the matrix B and the epilogue's staging tile.
//   q = 0 (targets 0..K-1): a tile is 128 consecutive tuples of 2^K adjacent
//       amplitudes: a 2D tensor map (row = tuple), boxes of 128 rows x 128 B
//       in the 128-byte swizzle, so a converter lane reading its row's
//       16-byte chunks meets the other lanes in distinct banks;
//   q >= 1: member m of tuple t sits at t_low + 2^q m + 2^(q+K) t_high; a 3D
//       map (low free bits, members, high free bits) with box
//       (min(2^(q+1), 256) floats, 2^K, 2^(7 - min(q, 7))): the lanes of a
//       warp read one member of 32 consecutive tuples, in runs of 2^min(q, 5)
//       lanes at consecutive addresses (2^(5-q)-way bank conflicts for q < 5;
//       at q = 1, 2 still faster than the register-fed kernel: 1.13 vs 1.6 ms
//       per 5-qubit block at n = 28).
// Warps 0-15 convert (warp w: TMEM lane quarter w mod 4, columns
// (W/4)(w/4) ..), 16-23 drain the accumulators as in k_block_tc, 24 issues
// the MMAs, 25 is the producer.  Every wait is bounded as in k_block_tc; the
// producer waits (bounded) for its last copies before the CTA exits.

constexpr int kTmaConvWarps = 16;
constexpr int kTmaConv = kTmaConvWarps * 32;                 // 512
constexpr int kTmaEpiWarp0 = kTmaConvWarps;                  // 16..23
constexpr int kTmaMmaWarp = kTmaConvWarps + kBkEpiWarps;     // 24
constexpr int kTmaProdWarp = kTmaMmaWarp + 1;                // 25
constexpr int kTmaThreads = (kTmaProdWarp + 1) * 32;         // 832
constexpr int kTmaRing = 4;                                  // raw tile stages

enum { TMA_ROWS = 0,     // q = 0: row-major tuples, 2D map, 128-byte swizzle
       TMA_MEMBERS = 1 };  // q >= 5: 3D map (low bits, members, high bits)

template <int K>
struct TmaSmem {
  static constexpr int D = 1 << K, W = 2 * D;
  static constexpr uint32_t RAW_BYTES = kTcRows * W * 4;     // 32 KB (K = 5)
  static constexpr uint32_t RAW0 = 0;                          // ring, 1024-aligned stages
  static constexpr uint32_t B_HI = kTmaRing * RAW_BYTES, B_LO = B_HI + W * W * 4;
  static constexpr uint32_t ROWOFF = B_LO + W * W * 4;
  static constexpr uint32_t DTAB = ROWOFF + kTcRows * 8;
  static constexpr uint32_t OFFS = DTAB + 4 * 256 * 8;
  // raw_full[R], raw_empty[R], afull[2], aempty[2], tfull[2], tempty[2], fin
  static constexpr uint32_t MBAR = OFFS + D * 4;
  static constexpr uint32_t FLAGS = MBAR + (2 * kTmaRing + 9) * 8;
  static constexpr int SROW = D + 2;
  static constexpr uint32_t STAGE = (FLAGS + 16 + 15) & ~15u;
  static constexpr uint32_t BYTES = STAGE + kTcRows * SROW * 8 + 1024;
  // tensor memory: accumulators at columns [0, 2W), A stages (hi | lo) at [2W, 6W)
  static constexpr uint32_t TCOLS = 6 * W <= 256 ? 256 : 512;
  __host__ __device__ static constexpr uint32_t a_col(int s) { return 2 * W + (uint32_t)s * 2 * W; }
};

template <int K>
struct TmaArgs {
  TcArgs<K> a;
  int q;       // lowest target
  int ql;      // min(q, 7): tuple-index bits below the targets inside a tile
};

__device__ __forceinline__ void mma_tf32_ta(uint32_t tmem_d, uint32_t tmem_a, uint64_t bdesc, uint32_t idesc,
                                            uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n\t}\n" ::"r"(tmem_d),
      "r"(tmem_a), "l"(bdesc), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t mbar, uint32_t bytes) {
  asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}\n" ::"r"(mbar),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const void* map, int x, int y, uint32_t mbar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(mbar)
      : "memory");
}

__device__ __forceinline__ void tma_load_3d(uint32_t dst, const void* map, int x, int y, int z, uint32_t mbar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(
          dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(mbar)
      : "memory");
}

// 32 lanes x N consecutive 32-bit TMEM columns from registers (thread i -> lane base + i)
template <int N>
__device__ __forceinline__ void tmem_st(uint32_t taddr, const float* v);
template <>
__device__ __forceinline__ void tmem_st<16>(uint32_t taddr, const float* v) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15, %16};\n" ::"r"(taddr),
      "f"(v[0]), "f"(v[1]), "f"(v[2]), "f"(v[3]), "f"(v[4]), "f"(v[5]), "f"(v[6]), "f"(v[7]), "f"(v[8]), "f"(v[9]),
      "f"(v[10]), "f"(v[11]), "f"(v[12]), "f"(v[13]), "f"(v[14]), "f"(v[15])
      : "memory");
}
template <>
__device__ __forceinline__ void tmem_st<8>(uint32_t taddr, const float* v) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};\n" ::"r"(taddr),
               "f"(v[0]), "f"(v[1]), "f"(v[2]), "f"(v[3]), "f"(v[4]), "f"(v[5]), "f"(v[6]), "f"(v[7])
               : "memory");
}

template <int K, int CASE>
__global__ void __launch_bounds__(kTmaThreads, 1)
k_block_tma(const __grid_constant__ TmaArgs<K> ta, const __grid_constant__ CUtensorMap map) {
  using L = TmaSmem<K>;
  constexpr int D = L::D, W = L::W;
  constexpr int CPW = W / 4;   // TMEM columns written per converter thread (16 or 8)
  const TcArgs<K>& a = ta.a;

  extern __shared__ unsigned char sm_raw[];
  unsigned char* sm = (unsigned char*)(((uintptr_t)sm_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* s_P = reinterpret_cast<uint64_t*>(sm + L::ROWOFF);
  uint32_t* s_off = reinterpret_cast<uint32_t*>(sm + L::OFFS);
  uint64_t* s_dtab = reinterpret_cast<uint64_t*>(sm + L::DTAB);
  const uint32_t mb0 = smem_u32(sm + L::MBAR);
  auto raw_full = [&](int r) { return mb0 + 8u * (uint32_t)r; };
  auto raw_empty = [&](int r) { return mb0 + 8u * (uint32_t)(kTmaRing + r); };
  auto afull = [&](int s) { return mb0 + 8u * (uint32_t)(2 * kTmaRing + s); };
  auto aempty = [&](int s) { return mb0 + 8u * (uint32_t)(2 * kTmaRing + 2 + s); };
  auto tfull = [&](int s) { return mb0 + 8u * (uint32_t)(2 * kTmaRing + 4 + s); };
  auto tempty = [&](int s) { return mb0 + 8u * (uint32_t)(2 * kTmaRing + 6 + s); };
  const uint32_t fin = mb0 + 8u * (uint32_t)(2 * kTmaRing + 8);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + L::FLAGS);
  volatile int* abort = reinterpret_cast<volatile int*>(sm + L::FLAGS + 4);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  // ---- setup: the matrix (hi / lo), offsets and tables for the epilogue, barriers, TMEM
  for (int e = tid; e < W * W; e += kTmaThreads) {
    const int n = e / W, kk = e % W;
    const float v = a.b[n][kk], h = tf32_hi(v);
    *reinterpret_cast<float*>(sm + L::B_HI + sw128_off(n, kk, W)) = h;
    *reinterpret_cast<float*>(sm + L::B_LO + sw128_off(n, kk, W)) = tf32_lo(v, h);
  }
  if (tid < D) s_off[tid] = a.off[tid];
  if (tid < kTcRows) s_P[tid] = row_offset(tid, a);
  for (int e = tid; e < 4 * 256; e += kTmaThreads) {
    const int c = e >> 8, sh = 7 + 8 * c;
    const uint64_t v = (uint64_t)(e & 255) << sh;
    s_dtab[e] = (sh < a.lg) ? deposit_nb(v & ((1ull << a.lg) - 1ull), a.s) : 0;
  }
  if (tid == 0) {
    for (int r = 0; r < kTmaRing; ++r) {
      mbar_init(raw_full(r), 1);
      mbar_init(raw_empty(r), kTmaConv);
    }
    for (int s = 0; s < 2; ++s) {
      mbar_init(afull(s), kTmaConv);
      mbar_init(aempty(s), 1);
      mbar_init(tfull(s), 1);
      mbar_init(tempty(s), (W / 32) * 4 * 32);
    }
    mbar_init(fin, 1);
    *abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == kTmaMmaWarp) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                 "r"(L::TCOLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tslot;
  const uint64_t stride_tiles = (uint64_t)gridDim.x;
  auto tile_row0 = [&](int i) { return ((uint64_t)blockIdx.x + (uint64_t)i * stride_tiles) * kTcRows; };
  auto tile_rows = [&](uint64_t t0) {
    return a.total - t0 < (uint64_t)kTcRows ? (int)(a.total - t0) : kTcRows;
  };

  if (warp < kTmaConvWarps) {
    // ================================================================ converters
    const int qd = warp & 3, cg = warp >> 2;
    const int t = qd * 32 + lane;            // this thread's tuple (row, TMEM lane)
    const int m0 = cg * (CPW / 2);           // first member of this thread
    uint32_t roff[CPW / 2];                  // byte offsets of the members inside a raw stage
#pragma unroll
    for (int j = 0; j < CPW / 2; ++j) {
      const int m = m0 + j;
      if (CASE == TMA_ROWS) {
        const int b = m >> 4, c16 = (m & 15) >> 1;
        roff[j] = (uint32_t)(b * kTcRows * 128 + t * 128 + ((c16 ^ (t & 7)) << 4) + (m & 1) * 8);
      } else {
        const int z = t >> ta.ql, x = t & ((1 << ta.ql) - 1);
        roff[j] = (uint32_t)((((z * D + m) << ta.ql) + x) * 8);
      }
    }
    const uint32_t lane_base = (uint32_t)(32 * qd) << 16;
    for (int i = 0; tile_row0(i) < a.total; ++i) {
      const int r = i % kTmaRing, s = i & 1;
      float v[CPW], lo[CPW];
      if (!mbar_wait(raw_full(r), (uint32_t)(i / kTmaRing) & 1u, abort)) break;
      const unsigned char* raw = sm + L::RAW0 + (uint32_t)r * L::RAW_BYTES;
#pragma unroll
      for (int j = 0; j < CPW / 2; ++j) {
        const float2 x = *reinterpret_cast<const float2*>(raw + roff[j]);
        v[2 * j] = x.x;
        v[2 * j + 1] = x.y;
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      mbar_arrive(raw_empty(r));
#pragma unroll
      for (int e = 0; e < CPW; ++e) {
        const float h = tf32_hi(v[e]);
        lo[e] = tf32_lo(v[e], h);
        v[e] = h;
      }
      // the A stage is free once the MMAs that read it two tiles ago have completed
      if (!mbar_wait(aempty(s), ((uint32_t)(i >> 1) & 1u) ^ 1u, abort)) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t col = L::a_col(s) + (uint32_t)(cg * CPW);
      tmem_st<CPW>(tmem + lane_base + col, v);
      tmem_st<CPW>(tmem + lane_base + col + W, lo);
      asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      mbar_arrive(afull(s));
    }
  } else if (warp < kTmaMmaWarp) {
    // ================================================================ epilogue (as in k_block_tc)
    const int e = warp - kTmaEpiWarp0;
    const int q = warp & 3;
    const int c = 32 * (e >> 2);
    const bool reads = c < W;
    const int t = q * 32 + lane;
    const int et = e * 32 + lane;
    const uint64_t myP = s_P[t];
    const bool staged = CASE == TMA_ROWS;   // rows are runs of 2^K >= 16 adjacent amplitudes
    float2* stage = reinterpret_cast<float2*>(sm + L::STAGE);
    for (int i = 0; tile_row0(i) < a.total; ++i) {
      const int s = i & 1;
      const uint64_t t0 = tile_row0(i);
      const int rows = tile_rows(t0);
      const bool valid = t < rows;
      const uint64_t tb = tile_base(t0, a, s_dtab);
      const uint64_t base = tb + myP;
      if (bar_or(2, kBkEpiThreads, !mbar_wait(tfull(s), (i >> 1) & 1, abort))) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      if (reads) {
        float y[32];
        tmem_ld32(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(s * W + c), y);
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        mbar_arrive(tempty(s));
        const int mm = c / 2;
        if (staged) {
#pragma unroll
          for (int m = 0; m < 16; m += 2)
            *reinterpret_cast<float4*>(stage + t * L::SROW + mm + m) =
                make_float4(y[2 * m], y[2 * m + 1], y[2 * m + 2], y[2 * m + 3]);
        } else if (valid) {
#pragma unroll
          for (int m = 0; m < 16; ++m) a.psi[base + s_off[mm + m]] = make_float2(y[2 * m], y[2 * m + 1]);
        }
      }
      if (staged) {
        bar_sync(2, kBkEpiThreads);
        constexpr int hb = K - 1;
#pragma unroll 4
        for (int k = 0; k < D / 4; ++k) {
          const int u = et + k * kBkEpiThreads;
          const int qq = (u & ((1 << hb) - 1)) | ((u >> (hb + 7)) << hb);
          const int tt = (u >> hb) & (kTcRows - 1);
          if (tt < rows)
            *reinterpret_cast<float4*>(a.psi + tb + s_P[tt] + s_off[2 * qq]) =
                *reinterpret_cast<const float4*>(stage + tt * L::SROW + 2 * qq);
        }
        bar_sync(2, kBkEpiThreads);
      }
    }
    __syncwarp();
  } else if (warp == kTmaMmaWarp) {
    // ================================================================ MMA issue (A from TMEM)
    if (lane == 0) {
      constexpr uint32_t idesc = tf32_idesc(W);
      const uint32_t b_hi = smem_u32(sm + L::B_HI), b_lo = smem_u32(sm + L::B_LO);
      bool issued = false;
      for (int i = 0; tile_row0(i) < a.total; ++i) {
        const int s = i & 1;
        const uint32_t ph = (uint32_t)(i >> 1) & 1u;
        if (!mbar_wait(afull(s), ph, abort)) break;
        if (!mbar_wait(tempty(s), ph ^ 1u, abort)) break;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t d = tmem + (uint32_t)(s * W);
        const uint32_t ahi = tmem + L::a_col(s), alo = ahi + W;
        // corrections first, then hi x hi (see k_block_tc)
#pragma unroll
        for (int pass = 0; pass < 2; ++pass)
#pragma unroll
          for (int ks = 0; ks < W / 8; ++ks) {
            const uint32_t koff = (uint32_t)(ks & 3) * 32u;
            const uint32_t bblk = (uint32_t)(ks >> 2) * (uint32_t)(W * 128);
            const uint64_t dbh = sw128_desc(b_hi + bblk + koff), dbl = sw128_desc(b_lo + bblk + koff);
            if (pass == 0) {
              mma_tf32_ta(d, ahi + 8u * ks, dbl, idesc, ks > 0 ? 1u : 0u);
              mma_tf32_ta(d, alo + 8u * ks, dbh, idesc, 1u);
            } else {
              mma_tf32_ta(d, ahi + 8u * ks, dbh, idesc, 1u);
            }
          }
        mma_commit(aempty(s));
        mma_commit(tfull(s));
        issued = true;
      }
      if (issued) {
        mma_commit(fin);
        volatile int never = 0;
        mbar_wait(fin, 0, &never);
      }
    }
    __syncwarp();
  } else {
    // ================================================================ producer (TMA)
    if (lane == 0) {
      asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&map)) : "memory");
      int issued = 0;
      for (int i = 0; tile_row0(i) < a.total; ++i) {
        const int r = i % kTmaRing;
        if (!mbar_wait(raw_empty(r), ((uint32_t)(i / kTmaRing) & 1u) ^ 1u, abort)) break;
        const uint32_t dst = smem_u32(sm + L::RAW0 + (uint32_t)r * L::RAW_BYTES);
        const uint64_t t0 = tile_row0(i);
        mbar_expect_tx(raw_full(r), L::RAW_BYTES);
        if (CASE == TMA_ROWS) {
#pragma unroll
          for (int b = 0; b < W / 32; ++b)
            tma_load_2d(dst + (uint32_t)b * kTcRows * 128, &map, 32 * b, (int)t0, raw_full(r));
        } else {
          const uint64_t low = t0 & ((1ull << ta.q) - 1ull);
          tma_load_3d(dst, &map, (int)(2 * low), 0, (int)(t0 >> ta.q), raw_full(r));
        }
        issued = i + 1;
      }
      // the last copies into every stage have landed before the CTA may exit
      volatile int never = 0;
      for (int j = issued > kTmaRing ? issued - kTmaRing : 0; j < issued; ++j)
        mbar_wait(raw_full(j % kTmaRing), (uint32_t)(j / kTmaRing) & 1u, &never);
    }
    __syncwarp();
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (tid == 0 && *abort) atomicExch(&g_tc_status, 1);
  if (warp == kTmaMmaWarp)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(L::TCOLS));
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_tiled() {
  static EncodeTiledFn fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(f);
    else
      cudaGetLastError();
  }
  return fn;
}

static int g_tma_enabled = 1;  // TMA-fed kernel for consecutive targets (QS_OPT_TENSOR_CORES >= 1)

// q: lowest target; the caller checked consecutive targets, no controls, a
// uniform batch, and 2^(n-K) >= 128 tuples per register.
template <int K>
static int launch_tma(const TcArgs<K>& a, int n, int nreg, int q, cudaStream_t st, bool* done) {
  using L = TmaSmem<K>;
  *done = false;
  EncodeTiledFn enc = encode_tiled();
  if (!enc) return QS_OK;
  TmaArgs<K> ta;
  ta.a = a;
  ta.q = q;
  ta.ql = std::min(q, 7);
  CUtensorMap map;
  memset(&map, 0, sizeof(map));
  const uint64_t tuples = (uint64_t)nreg << (n - K);
  CUresult rc;
  if (q == 0) {
    if (tuples >= (1ull << 31)) return QS_OK;
    const cuuint64_t dims[2] = {(cuuint64_t)(2 << K), (cuuint64_t)tuples};
    const cuuint64_t strides[1] = {(cuuint64_t)(8u << K)};
    const cuuint32_t box[2] = {32, (cuuint32_t)kTcRows};
    const cuuint32_t es[2] = {1, 1};
    rc = enc(&map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, (void*)a.psi, dims, strides, box, es,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  } else {
    if (q < 1 || q > 30 || q + K > n) return QS_OK;
    const uint64_t high = tuples >> q;   // free-bit combinations above the targets, over all registers
    if (high >= (1ull << 31)) return QS_OK;
    const int ql = std::min(q, 7);
    const cuuint64_t dims[3] = {(cuuint64_t)(2ull << q), (cuuint64_t)(1u << K), (cuuint64_t)high};
    const cuuint64_t strides[2] = {(cuuint64_t)(8ull << q), (cuuint64_t)(8ull << (q + K))};
    const cuuint32_t box[3] = {(cuuint32_t)std::min(2 << ql, 256), (cuuint32_t)(1u << K), (cuuint32_t)(1u << (7 - ql))};
    const cuuint32_t es[3] = {1, 1, 1};
    rc = enc(&map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, (void*)a.psi, dims, strides, box, es,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  }
  if (rc != CUDA_SUCCESS) return QS_OK;   // not expressible as a tensor map: the register-fed kernel runs
  int dev = 0, sms = 0;
  QS_CUDA(cudaGetDevice(&dev));
  QS_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const size_t smem = L::BYTES;
  const uint64_t tiles = (a.total + kTcRows - 1) / kTcRows;
  const unsigned grid = (unsigned)std::min<uint64_t>(tiles, (uint64_t)sms);
  if (q == 0) {
    QS_CUDA(cudaFuncSetAttribute(k_block_tma<K, TMA_ROWS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_block_tma<K, TMA_ROWS><<<grid, kTmaThreads, smem, st>>>(ta, map);
  } else {
    QS_CUDA(cudaFuncSetAttribute(k_block_tma<K, TMA_MEMBERS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_block_tma<K, TMA_MEMBERS><<<grid, kTmaThreads, smem, st>>>(ta, map);
  }
  QS_LAUNCHED();
  *done = true;
  return QS_OK;
}

template <int K>
static int launch_tc_t(float2* psi, int n, int nreg, const Plan& p, cudaStream_t st) {
  constexpr int D = 1 << K;
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
      a.b[2 * r][2 * c] = ur;
      a.b[2 * r][2 * c + 1] = -ui;
      a.b[2 * r + 1][2 * c] = ui;
      a.b[2 * r + 1][2 * c + 1] = ur;
    }
  QS_TRY(make_idx(n, locmask | p.ctrl_mask, p.ctrl_vals, &a.s));
  a.psi = psi;
  a.lg = a.s.item_log2;
  a.reg_stride = 1ull << n;
  a.total = (1ull << a.lg) * (uint64_t)nreg;
  if (a.total == 0) return QS_OK;
  {
    const int q = p.locs[order[0]];
    const bool consecutive = p.locs[order[K - 1]] == q + K - 1;
    if (g_tma_enabled && consecutive && p.ctrl_mask == 0 && n - K >= 7) {
      bool done = false;
      QS_TRY(launch_tma<K>(a, n, nreg, q, st, &done));
      if (done) return QS_OK;
    }
  }
  if (a.lowbits >= 1) return launch_tc_mode<K, TC_PAIR_MEMBERS>(a, st);
  if (!(p.ctrl_mask & 1ull) && a.lg >= 1) return launch_tc_mode<K, TC_PAIR_TUPLES>(a, st);
  return launch_tc_mode<K, TC_SCALAR>(a, st);
}

// ------------------------------------------------------------------ Gram matrix on the tensor cores
//
// G = sum over the tuples x of a k-qubit support (k = 4, 5) of psi_x^T lambda_x
// in the interleaved real form (row / column 2m = Re, 2m + 1 = Im of member m),
// the one pass of the block backward that forms rho = sum_x psi_x lambda_x^dag.
// A 128-tuple tile is staged transposed: rows are components (psi in rows
// 0..63, lambda in rows 64..127, 4-qubit supports zero-padded), columns are the
// tuples, in the K-major 128-byte-swizzle layout (kind::tf32 takes K-major
// operands only).  One tcgen05.mma (M = 64, N = 2^(K+1), K = 8 tuples) takes
// A = rows 0..63 (psi^T) and B = rows 64.. (lambda^T): the accumulator is
// psi^T lambda (an M = 128 MMA over rows 0..127 would spend half its work on
// lambda^T lambda).  3xTF32 as in k_block_tc; FP32
// accumulation in TMEM over groups of 8 tiles, flushed by the epilogue warps
// into an FP64 matrix in shared memory, written per CTA for a fixed-order fold.

constexpr int kGramGroup = 8;  // tiles per FP32 accumulation group

template <int K>
struct GramTcSmem {
  static constexpr uint32_t T_BYTES = kTcRows * 128 * 4;   // 128 x 128 fp32: 64 KB
  static constexpr uint32_t HI = 0, LO = T_BYTES;
  static constexpr uint32_t ROWOFF = 2 * T_BYTES;
  static constexpr uint32_t DTAB = ROWOFF + kTcRows * 8;
  static constexpr uint32_t OFFS = DTAB + 4 * 256 * 8;
  static constexpr uint32_t ACC = OFFS + 64 * 4;            // FP64 [64][65]
  static constexpr int ACC_LD = 65;
  static constexpr uint32_t MBAR = ACC + 64 * ACC_LD * 8;   // full, empty, tfull[2], tempty[2], fin
  static constexpr uint32_t FLAGS = MBAR + 7 * 8;
  static constexpr uint32_t BYTES = FLAGS + 16 + 1024;
};

template <int K, int MODE>
__global__ void __launch_bounds__(kTcThreads, 1) k_gram_tc(const __grid_constant__ TcArgs<K> a, const float2* lam,
                                                           double* partials) {
  using L = GramTcSmem<K>;
  constexpr int D = 1 << K, W = 2 * D;   // components per state
  constexpr int NU = MODE == TC_SCALAR ? kTcRows * D : kTcRows * D / 2;
  constexpr int UT = NU / kTcLoaders;
  static_assert(UT * kTcLoaders == NU && UT <= 8, "tile splits evenly over the loaders");
  using VT = typename std::conditional<MODE == TC_SCALAR, float2, float4>::type;
  extern __shared__ unsigned char sm_raw[];
  unsigned char* sm = (unsigned char*)(((uintptr_t)sm_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* s_P = reinterpret_cast<uint64_t*>(sm + L::ROWOFF);
  uint64_t* s_dtab = reinterpret_cast<uint64_t*>(sm + L::DTAB);
  uint32_t* s_off = reinterpret_cast<uint32_t*>(sm + L::OFFS);
  double* acc = reinterpret_cast<double*>(sm + L::ACC);
  const uint32_t mb0 = smem_u32(sm + L::MBAR);
  const uint32_t full = mb0, empty = mb0 + 8u, fin = mb0 + 48u;
  auto tfull = [&](int b) { return mb0 + 16u + 8u * (uint32_t)b; };
  auto tempty = [&](int b) { return mb0 + 32u + 8u * (uint32_t)b; };
  uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + L::FLAGS);
  volatile int* abort = reinterpret_cast<volatile int*>(sm + L::FLAGS + 4);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  // ---- setup: zeroed tiles (4-qubit supports leave columns unused), FP64
  // accumulator, offsets, tables, barriers, TMEM
  for (uint32_t e = tid; e < 2 * L::T_BYTES / 16; e += kTcThreads)
    reinterpret_cast<float4*>(sm + L::HI)[e] = make_float4(0.f, 0.f, 0.f, 0.f);
  for (int e = tid; e < 64 * L::ACC_LD; e += kTcThreads) acc[e] = 0.0;
  if (tid < D) s_off[tid] = a.off[tid];
  if (tid < kTcRows) s_P[tid] = row_offset(tid, a);
  for (int e = tid; e < 4 * 256; e += kTcThreads) {
    const int c = e >> 8, sh = 7 + 8 * c;
    const uint64_t v = (uint64_t)(e & 255) << sh;
    s_dtab[e] = (sh < a.lg) ? deposit_nb(v & ((1ull << a.lg) - 1ull), a.s) : 0;
  }
  if (tid == 0) {
    mbar_init(full, kTcLoaders);
    mbar_init(empty, 1);
    for (int b = 0; b < 2; ++b) {
      mbar_init(tfull(b), 1);
      mbar_init(tempty(b), kTcEpiWarps * 32);
    }
    mbar_init(fin, 1);
    *abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == kTcMmaWarp) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                 "r"(128u));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tslot;
  const uint64_t stride_tiles = (uint64_t)gridDim.x;
  auto tile_row0 = [&](int i) { return ((uint64_t)blockIdx.x + (uint64_t)i * stride_tiles) * kTcRows; };
  auto tile_rows = [&](uint64_t t0) {
    return a.total - t0 < (uint64_t)kTcRows ? (int)(a.total - t0) : kTcRows;
  };
  int ntiles = 0;
  while (tile_row0(ntiles) < a.total) ++ntiles;
  const int ngroups = (ntiles + kGramGroup - 1) / kGramGroup;

  if (warp < kTcLoadWarps) {
    // ================================================================ loaders (psi and lambda)
    const int lt = tid, lb = a.lowbits;
    uint64_t goff[UT];
    uint32_t tm[UT];  // the unit's tuple t (bits 0..7) and first member m (bits 8..)
    int tmax = 0;
#pragma unroll
    for (int k = 0; k < UT; ++k) {
      const int u = lt + k * kTcLoaders;
      int t, m;
      if (MODE == TC_PAIR_MEMBERS) {
        const int hb = lb - 1;
        t = (u >> hb) & (kTcRows - 1);
        m = 2 * ((u & ((1 << hb) - 1)) | ((u >> (hb + 7)) << hb));
      } else if (MODE == TC_PAIR_TUPLES) {
        t = 2 * (u & (kTcRows / 2 - 1));
        m = u >> 6;
      } else {
        t = u & (kTcRows - 1);
        m = u >> 7;
      }
      goff[k] = s_P[t] + s_off[m];
      tm[k] = (uint32_t)t | ((uint32_t)m << 8);
      tmax = max(tmax, MODE == TC_PAIR_TUPLES ? t + 1 : t);
    }
    VT p0[UT], l0[UT], p1[UT], l1[UT];
    auto load = [&](uint64_t t0, VT* vp, VT* vl) {
      const uint64_t tb = tile_base(t0, a, s_dtab);
      const int rows = tile_rows(t0);
#pragma unroll
      for (int k = 0; k < UT; ++k) {
        const int t = (int)(tm[k] & 255u);
        const bool ok = tmax < rows || t < rows;
        vp[k] = ok ? *reinterpret_cast<const VT*>(a.psi + tb + goff[k]) : VT{};
        vl[k] = ok ? *reinterpret_cast<const VT*>(lam + tb + goff[k]) : VT{};
      }
    };
    // transposed staging: component row r (psi r, lambda 64 + r), tuple column t
    auto put1 = [&](int r, int t, float v) {
      const uint32_t o = sw128_off(r, t, kTcRows);
      const float h = tf32_hi(v);
      *reinterpret_cast<float*>(sm + L::HI + o) = h;
      *reinterpret_cast<float*>(sm + L::LO + o) = tf32_lo(v, h);
    };
    auto put2 = [&](int r, int t, float v0, float v1) {  // columns t, t + 1 (t even): one 8-byte store
      const uint32_t o = sw128_off(r, t, kTcRows);
      const float h0 = tf32_hi(v0), h1 = tf32_hi(v1);
      *reinterpret_cast<float2*>(sm + L::HI + o) = make_float2(h0, h1);
      *reinterpret_cast<float2*>(sm + L::LO + o) = make_float2(tf32_lo(v0, h0), tf32_lo(v1, h1));
    };
    auto put = [&](int r0, uint32_t tmk, const VT& x) {
      const int t = (int)(tmk & 255u), m = (int)(tmk >> 8);
      if (MODE == TC_PAIR_MEMBERS) {  // members m, m + 1 of tuple t
        const float4 v = *reinterpret_cast<const float4*>(&x);
        put1(r0 + 2 * m, t, v.x);
        put1(r0 + 2 * m + 1, t, v.y);
        put1(r0 + 2 * m + 2, t, v.z);
        put1(r0 + 2 * m + 3, t, v.w);
      } else if (MODE == TC_PAIR_TUPLES) {  // member m of tuples t, t + 1
        const float4 v = *reinterpret_cast<const float4*>(&x);
        put2(r0 + 2 * m, t, v.x, v.z);
        put2(r0 + 2 * m + 1, t, v.y, v.w);
      } else {
        const float2 v = *reinterpret_cast<const float2*>(&x);
        put1(r0 + 2 * m, t, v.x);
        put1(r0 + 2 * m + 1, t, v.y);
      }
    };
    auto step = [&](int i, const VT* cp, const VT* cl, VT* np, VT* nl) -> bool {
      if (i >= ntiles) return false;
      if (i + 1 < ntiles) load(tile_row0(i + 1), np, nl);
      if (!mbar_wait(empty, (uint32_t)(i & 1) ^ 1u, abort)) return false;  // the previous tile's MMAs are done
#pragma unroll
      for (int k = 0; k < UT; ++k) {
        put(0, tm[k], cp[k]);
        put(64, tm[k], cl[k]);
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      mbar_arrive(full);
      return true;
    };
    if (ntiles > 0) load(tile_row0(0), p0, l0);
    for (int i = 0;; i += 2) {
      if (!step(i, p0, l0, p1, l1)) break;
      if (!step(i + 1, p1, l1, p0, l0)) break;
    }
  } else if (warp < kTcMmaWarp) {
    // ================================================================ epilogue: FP32 groups into FP64
    const int q = warp - kTcEpiWarp0;
    // M = 64 accumulator: row r sits in TMEM lane 32 (r / 16) + r mod 16 (measured on
    // GB300), so lanes 0..15 of every lane quarter hold rows 16 q .. 16 q + 15
    const int row = 16 * q + lane;
    const bool valid_row = lane < 16 && row < W;
    for (int g = 0; g < ngroups; ++g) {
      const int b = g & 1;
      if (!__all_sync(0xffffffffu, mbar_wait(tfull(b), (uint32_t)(g >> 1) & 1u, abort))) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      // 32 columns at a time into the FP64 row; the buffer is released after the last
#pragma unroll
      for (int c0 = 0; c0 < W; c0 += 32) {
        float y[32];
        tmem_ld32(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(b * 64 + c0), y);
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        if (c0 + 32 == W) {
          asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
          mbar_arrive(tempty(b));
        }
        if (valid_row) {
#pragma unroll
          for (int c = 0; c < 32; ++c) acc[row * L::ACC_LD + c0 + c] += (double)y[c];
        }
      }
    }
    __syncwarp();
  } else {
    // ================================================================ MMA issue
    if (lane == 0) {
      // D (64 x W) = psi^T (rows 0..63) x lambda^T (rows 64..64+W-1): M = 64, N = W
      constexpr uint32_t idesc = tf32_idesc(W, 64);
      const uint32_t base_hi = smem_u32(sm + L::HI), base_lo = smem_u32(sm + L::LO);
      const uint32_t lam_off = 64u * 128u;  // lambda: rows 64.. of every 128-row column block
      bool issued = false;
      for (int i = 0; i < ntiles; ++i) {
        const int g = i / kGramGroup, b = g & 1;
        if (!mbar_wait(full, (uint32_t)i & 1u, abort)) break;
        if (i % kGramGroup == 0 && !mbar_wait(tempty(b), ((uint32_t)(g >> 1) & 1u) ^ 1u, abort)) break;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t d = tmem + (uint32_t)(b * 64);
        // corrections first, then hi x hi (fewer truncating passes of the large terms)
#pragma unroll
        for (int pass = 0; pass < 2; ++pass)
#pragma unroll
          for (int ks = 0; ks < kTcRows / 8; ++ks) {
            // 8 tuples per MMA: 32 bytes inside a 128-byte column block of 32 tuples
            const uint32_t ko = (uint32_t)(ks >> 2) * (uint32_t)(kTcRows * 128) + (uint32_t)(ks & 3) * 32u;
            const uint64_t ah = sw128_desc(base_hi + ko), al = sw128_desc(base_lo + ko);
            const uint64_t bh = sw128_desc(base_hi + lam_off + ko), bl = sw128_desc(base_lo + lam_off + ko);
            if (pass == 0) {
              mma_tf32(d, ah, bl, idesc, (i % kGramGroup != 0 || ks > 0) ? 1u : 0u);
              mma_tf32(d, al, bh, idesc, 1u);
            } else {
              mma_tf32(d, ah, bh, idesc, 1u);
            }
          }
        mma_commit(empty);
        if (i % kGramGroup == kGramGroup - 1 || i == ntiles - 1) mma_commit(tfull(b));
        issued = true;
      }
      if (issued) {
        mma_commit(fin);
        volatile int never = 0;
        mbar_wait(fin, 0, &never);
      }
    }
    __syncwarp();
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (tid == 0 && *abort) atomicExch(&g_tc_status, 1);
  for (int e = tid; e < W * W; e += kTcThreads)
    partials[(size_t)blockIdx.x * W * W + e] = acc[(e / W) * L::ACC_LD + (e % W)];
  if (warp == kTcMmaWarp) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(128u));
}

template <int K, int MODE>
static int launch_gram_tc_mode(const TcArgs<K>& a, const float2* lam, double* partials, int* grid_out,
                               cudaStream_t st) {
  using L = GramTcSmem<K>;
  int dev = 0, sms = 0;
  QS_CUDA(cudaGetDevice(&dev));
  QS_CUDA(cudaFuncSetAttribute(k_gram_tc<K, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L::BYTES));
  QS_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const uint64_t tiles = (a.total + kTcRows - 1) / kTcRows;
  const unsigned grid = (unsigned)std::min<uint64_t>(tiles, (uint64_t)sms);
  k_gram_tc<K, MODE><<<grid, kTcThreads, L::BYTES, st>>>(a, lam, partials);
  QS_LAUNCHED();
  *grid_out = (int)grid;
  return QS_OK;
}

template <int K>
static int launch_gram_tc_t(const float2* psi, const float2* lam, int n, const int* qubits, double* partials,
                            int* grid_out, cudaStream_t st) {
  constexpr int D = 1 << K;
  TcArgs<K> a;
  memset(&a, 0, sizeof(a));
  uint64_t mask = 0;
  for (int j = 0; j < K; ++j) mask |= 1ull << qubits[j];
  a.lowbits = 0;
  while (a.lowbits < K && qubits[a.lowbits] == a.lowbits) ++a.lowbits;
  for (int m = 0; m < D; ++m) {
    uint64_t o = 0;
    for (int j = 0; j < K; ++j)
      if ((m >> j) & 1) o |= 1ull << qubits[j];
    if (o >> 32) return fail(QS_EUNSUPPORTED, "tensor-core Gram takes supports below qubit 32");
    a.off[m] = (uint32_t)o;
  }
  QS_TRY(make_idx(n, mask, 0, &a.s));
  a.psi = const_cast<float2*>(psi);
  a.lg = a.s.item_log2;
  a.reg_stride = 1ull << n;
  a.total = 1ull << a.lg;
  if (a.lowbits >= 1) return launch_gram_tc_mode<K, TC_PAIR_MEMBERS>(a, lam, partials, grid_out, st);
  if (a.lg >= 1) return launch_gram_tc_mode<K, TC_PAIR_TUPLES>(a, lam, partials, grid_out, st);
  return launch_gram_tc_mode<K, TC_SCALAR>(a, lam, partials, grid_out, st);
}

// ------------------------------------------------------------------ TMA-fed Gram on consecutive supports
//
// The same Gram matrix for supports q..q+K-1 with the loads done by TMA: a
// producer thread copies each 32-tuple tile of psi and of lambda into a
// four-stage ring (the register-held loads of k_gram_tc, 64 KB in flight per
// SM, bound it to about 3 TB/s), sixteen converter warps write it transposed
// and split (hi / lo) into one of four operand stages (a warp step writes one
// 32-byte-swizzle K step: 4 components x 8 tuples).  A = [psi_hi^T; psi_lo^T]
// fills all M = 128 rows, and two MMAs per 8 tuples (B = lambda_hi^T, then
// lambda_lo^T) give rows r + rows r + 64 = psi^T lambda to FP32 accuracy.
// Measured alternatives (n = 28 brickwork gradient 0.179 s with this form):
// one N = 128 MMA over B = [lambda_hi^T; lambda_lo^T] instead of two N = 64
// ones 0.188 s; rings of 6 or 8 stages with 3 or 2 operand stages unchanged;
// A in tensor memory issues no faster than A in shared memory (an issue loop
// of M = 128, N = 64, K = 8 tf32 MMAs: ~94 cycles each either way).  Raw
// layouts as in k_block_tma: q = 0 row-major tuples (2D map, 128-byte
// swizzle), q >= 1 members x tuples (3D map; box (min(2^(q+1), 64) floats,
// 2^K, 2^(5 - min(q, 5)))).
constexpr int kGtTuples = 32;
constexpr int kGtRing = 4;
constexpr int kGtStages = 4;                     // operand stages (MMA completion runs several tiles behind)
constexpr int kGtGroup = 32;                     // tiles per FP32 accumulation group (1024 tuples)
constexpr int kGtConvWarps = 16;
constexpr int kGtConv = kGtConvWarps * 32;
constexpr int kGtEpiWarp0 = kGtConvWarps;        // 16..19
constexpr int kGtMmaWarp = kGtConvWarps + 4;     // 20
constexpr int kGtProdWarp = kGtMmaWarp + 1;      // 21
constexpr int kGtThreads = (kGtProdWarp + 1) * 32;

template <int K>
struct GramTmaSmem {
  static constexpr int D = 1 << K, W = 2 * D;
  static constexpr uint32_t RAW_STATE = kGtTuples * W * 4;               // one state's tile: 8 KB (K = 5)
  static constexpr uint32_t RAW_STAGE = 2 * RAW_STATE;                   // psi then lambda
  static constexpr uint32_t OP_BYTES = kTcRows * kGtTuples * 4;          // 128 rows x 32 tuples: 16 KB
  static constexpr uint32_t RAW0 = 0;
  __host__ __device__ static constexpr uint32_t raw(int r) { return RAW0 + (uint32_t)r * 16384u; }
  // stage s: A = [psi_hi^T; psi_lo^T] at op_a(s), B = [lambda_hi^T; lambda_lo^T] after it
  static constexpr uint32_t OP0 = kGtRing * 16384u;
  static constexpr uint32_t OP_END = OP0 + kGtStages * 2 * OP_BYTES;
  __host__ __device__ static constexpr uint32_t op_a(int s) { return OP0 + (uint32_t)s * 2 * OP_BYTES; }
  static constexpr uint32_t ACC = OP_END;                                // FP64 [64][65]
  static constexpr int ACC_LD = 65;
  // raw_full[R], raw_empty[R], op_full[S], op_empty[S], tfull[2], tempty[2], fin
  static constexpr uint32_t MBAR = ACC + 64 * ACC_LD * 8;
  static constexpr uint32_t FLAGS = MBAR + (2 * kGtRing + 2 * kGtStages + 5) * 8;
  static constexpr uint32_t BYTES = FLAGS + 16 + 1024;
};

template <int K, int CASE>
__global__ void __launch_bounds__(kGtThreads, 1)
k_gram_tma(const __grid_constant__ CUtensorMap map_psi, const __grid_constant__ CUtensorMap map_lam, uint64_t total,
           int q, double* partials) {
  using L = GramTmaSmem<K>;
  constexpr int D = L::D, W = L::W;
  constexpr int GT = kGtTuples;
  extern __shared__ unsigned char sm_raw[];
  unsigned char* sm = (unsigned char*)(((uintptr_t)sm_raw + 1023) & ~(uintptr_t)1023);
  double* acc = reinterpret_cast<double*>(sm + L::ACC);
  const uint32_t mb0 = smem_u32(sm + L::MBAR);
  auto raw_full = [&](int r) { return mb0 + 8u * (uint32_t)r; };
  auto raw_empty = [&](int r) { return mb0 + 8u * (uint32_t)(kGtRing + r); };
  auto op_full = [&](int s) { return mb0 + 8u * (uint32_t)(2 * kGtRing + s); };
  auto op_empty = [&](int s) { return mb0 + 8u * (uint32_t)(2 * kGtRing + kGtStages + s); };
  auto tfull = [&](int b) { return mb0 + 8u * (uint32_t)(2 * kGtRing + 2 * kGtStages + b); };
  auto tempty = [&](int b) { return mb0 + 8u * (uint32_t)(2 * kGtRing + 2 * kGtStages + 2 + b); };
  const uint32_t fin = mb0 + 8u * (uint32_t)(2 * kGtRing + 2 * kGtStages + 4);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + L::FLAGS);
  volatile int* abort = reinterpret_cast<volatile int*>(sm + L::FLAGS + 4);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int ql = q < 5 ? q : 5;

  // ---- setup: zero operand stages (4-qubit supports leave rows unused), FP64 accumulator, barriers, TMEM
  for (uint32_t e = tid; e < kGtStages * 2 * L::OP_BYTES / 16; e += kGtThreads)
    reinterpret_cast<float4*>(sm + L::OP0)[e] = make_float4(0.f, 0.f, 0.f, 0.f);
  for (int e = tid; e < 64 * L::ACC_LD; e += kGtThreads) acc[e] = 0.0;
  if (tid == 0) {
    for (int r = 0; r < kGtRing; ++r) {
      mbar_init(raw_full(r), 1);
      mbar_init(raw_empty(r), kGtConvWarps);
    }
    for (int r = 0; r < kGtStages; ++r) {
      mbar_init(op_full(r), kGtConvWarps);
      mbar_init(op_empty(r), 1);
    }
    for (int r = 0; r < 2; ++r) {
      mbar_init(tfull(r), 1);
      mbar_init(tempty(r), 4 * 32);
    }
    mbar_init(fin, 1);
    *abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == kGtMmaWarp) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                 "r"(128u));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tslot;
  const uint64_t stride_tiles = (uint64_t)gridDim.x;
  auto tile_t0 = [&](int i) { return ((uint64_t)blockIdx.x + (uint64_t)i * stride_tiles) * GT; };
  int ntiles = 0;
  while (tile_t0(ntiles) < total) ++ntiles;
  const int ngroups = (ntiles + kGtGroup - 1) / kGtGroup;

  if (warp < kGtConvWarps) {
    // ================================================================ converters
    // unit u = warp + 16 j (j < 8): state (psi / lambda), 4 components c0..c0+3 and one K
    // step of 8 tuples; lane = 8 (component offset) + tuple offset.  A warp writes the
    // hi rows c0..c0+3 (one 128-byte run) and the lo rows 64 + c0.. of its state's operand.
    const int lc = lane >> 3, lt = lane & 7;
    for (int i = 0; i < ntiles; ++i) {
      const int r0 = i % kGtRing, s = i % kGtStages;
      if (!mbar_wait(raw_full(r0), (uint32_t)(i / kGtRing) & 1u, abort)) break;
      const unsigned char* raw = sm + L::raw(r0);
      float v[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int u = warp + 16 * j;               // 0..127
        const int st = u >> 6, cg = (u >> 2) & 15, ks = u & 3;
        const int c = 4 * cg + lc, t = 8 * ks + lt;
        float x = 0.f;
        if (c < W) {
          const unsigned char* sp = raw + (st ? L::RAW_STATE : 0u);
          uint32_t o;
          if (CASE == TMA_ROWS) {
            const int bb = c >> 5, c16 = (c & 31) >> 2;
            o = (uint32_t)(bb * GT * 128 + t * 128 + ((c16 ^ (t & 7)) << 4) + (c & 3) * 4);
          } else {
            const int z = t >> ql, xx = t & ((1 << ql) - 1);
            o = (uint32_t)(((((z * D + (c >> 1)) << ql) + xx) * 2 + (c & 1)) * 4);
          }
          x = *reinterpret_cast<const float*>(sp + o);
        }
        v[j] = x;
      }
      // one arrival per warp: its lanes' reads are ordered before lane 0's arrive
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(raw_empty(r0));
      // the operand stage is free once the MMAs of tile i - kGtStages have completed
      if (!mbar_wait(op_empty(s), ((uint32_t)(i / kGtStages) & 1u) ^ 1u, abort)) break;
      unsigned char* oa = sm + L::op_a(s);
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int u = warp + 16 * j;
        const int st = u >> 6, cg = (u >> 2) & 15, ks = u & 3;
        const int c = 4 * cg + lc, t = 8 * ks + lt;
        if (c >= W) continue;
        unsigned char* ob = oa + (st ? L::OP_BYTES : 0u);
        const float hv = tf32_hi(v[j]);
        *reinterpret_cast<float*>(ob + sw32_off(c, t, kTcRows)) = hv;
        *reinterpret_cast<float*>(ob + sw32_off(64 + c, t, kTcRows)) = tf32_lo(v[j], hv);
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(op_full(s));
    }
  } else if (warp < kGtMmaWarp) {
    // ================================================================ epilogue: FP32 groups into FP64
    // M = 128 accumulator: TMEM lane r = row r; rows r (psi_hi) and r + 64 (psi_lo)
    // both add into component r, the lo half after the hi half (named barrier 3)
    const int qd = warp - kGtEpiWarp0;
    const int row = (32 * qd + lane) & 63;
    const bool valid_row = row < W;
    for (int g = 0; g < ngroups; ++g) {
      const int b = g & 1;
      // the four epilogue warps agree on giving up (they share named barrier 3)
      if (bar_or(3, 4 * 32, !mbar_wait(tfull(b), (uint32_t)(g >> 1) & 1u, abort))) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
      for (int cc = 0; cc < W / 32; ++cc) {
        float y[32];
        tmem_ld32(tmem + ((uint32_t)(32 * qd) << 16) + (uint32_t)(b * 64 + 32 * cc), y);
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        if (cc == W / 32 - 1) {
          asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
          mbar_arrive(tempty(b));
        }
        for (int half = 0; half < 2; ++half) {
          if ((qd >> 1) == half && valid_row) {
#pragma unroll
            for (int c = 0; c < 32; ++c) acc[row * L::ACC_LD + 32 * cc + c] += (double)y[c];
          }
          bar_sync(3, 4 * 32);
        }
      }
    }
    __syncwarp();
  } else if (warp == kGtMmaWarp) {
    // ================================================================ MMA issue
    if (lane == 0) {
      constexpr uint32_t idesc = tf32_idesc(W);   // M = 128, N = W
      const uint32_t lo_off = 64u * 32u;           // rows 64.. inside every K step's block
      bool issued = false;
      for (int i = 0; i < ntiles; ++i) {
        const int g = i / kGtGroup, b = g & 1, s = i % kGtStages;
        if (!mbar_wait(op_full(s), (uint32_t)(i / kGtStages) & 1u, abort)) break;
        if (i % kGtGroup == 0 && !mbar_wait(tempty(b), ((uint32_t)(g >> 1) & 1u) ^ 1u, abort)) break;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t base_a = smem_u32(sm + L::op_a(s)), base_b = base_a + L::OP_BYTES;
        const uint32_t d = tmem + (uint32_t)(b * 64);
        // the lambda_lo products first, then lambda_hi (fewer truncating passes of the large terms)
#pragma unroll
        for (int pass = 0; pass < 2; ++pass)
#pragma unroll
          for (int ks = 0; ks < GT / 8; ++ks) {
            const uint32_t ko = (uint32_t)ks * (uint32_t)(kTcRows * 32);   // K step: 128 rows x 32 bytes
            const uint64_t da = sw32_desc(base_a + ko);
            const uint64_t bh = sw32_desc(base_b + ko), bl = sw32_desc(base_b + lo_off + ko);
            if (pass == 0) mma_tf32(d, da, bl, idesc, (i % kGtGroup != 0 || ks > 0) ? 1u : 0u);
            else mma_tf32(d, da, bh, idesc, 1u);
          }
        mma_commit(op_empty(s));
        if (i % kGtGroup == kGtGroup - 1 || i == ntiles - 1) mma_commit(tfull(b));
        issued = true;
      }
      if (issued) {
        mma_commit(fin);
        volatile int never = 0;
        mbar_wait(fin, 0, &never);
      }
    }
    __syncwarp();
  } else {
    // ================================================================ producer (TMA, psi and lambda)
    if (lane == 0) {
      asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&map_psi)) : "memory");
      asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&map_lam)) : "memory");
      int issued = 0;
      for (int i = 0; i < ntiles; ++i) {
        const int r = i % kGtRing;
        if (!mbar_wait(raw_empty(r), ((uint32_t)(i / kGtRing) & 1u) ^ 1u, abort)) break;
        const uint32_t dst = smem_u32(sm + L::raw(r));
        const uint64_t t0 = tile_t0(i);
        mbar_expect_tx(raw_full(r), L::RAW_STAGE);
        if (CASE == TMA_ROWS) {
#pragma unroll
          for (int b = 0; b < W / 32; ++b) {
            tma_load_2d(dst + (uint32_t)b * GT * 128, &map_psi, 32 * b, (int)t0, raw_full(r));
            tma_load_2d(dst + L::RAW_STATE + (uint32_t)b * GT * 128, &map_lam, 32 * b, (int)t0, raw_full(r));
          }
        } else {
          const uint64_t low = t0 & ((1ull << q) - 1ull);
          tma_load_3d(dst, &map_psi, (int)(2 * low), 0, (int)(t0 >> q), raw_full(r));
          tma_load_3d(dst + L::RAW_STATE, &map_lam, (int)(2 * low), 0, (int)(t0 >> q), raw_full(r));
        }
        issued = i + 1;
      }
      volatile int never = 0;
      for (int j = issued > kGtRing ? issued - kGtRing : 0; j < issued; ++j)
        mbar_wait(raw_full(j % kGtRing), (uint32_t)(j / kGtRing) & 1u, &never);
    }
    __syncwarp();
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (tid == 0 && *abort) atomicExch(&g_tc_status, 1);
  for (int e = tid; e < W * W; e += kGtThreads)
    partials[(size_t)blockIdx.x * W * W + e] = acc[(e / W) * L::ACC_LD + (e % W)];
  if (warp == kGtMmaWarp) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(128u));
}

// psi and lambda tensor maps of one register for a consecutive support q..q+K-1
// (the same geometry as k_block_tma's, with 64-tuple boxes); false if not expressible
template <int K>
static bool gram_maps(const float2* psi, const float2* lam, int n, int q, CUtensorMap* mp, CUtensorMap* ml) {
  EncodeTiledFn enc = encode_tiled();
  if (!enc) return false;
  const uint64_t tuples = 1ull << (n - K);
  for (int which = 0; which < 2; ++which) {
    CUtensorMap* map = which ? ml : mp;
    void* base = (void*)(which ? lam : psi);
    memset(map, 0, sizeof(*map));
    CUresult rc;
    if (q == 0) {
      const cuuint64_t dims[2] = {(cuuint64_t)(2 << K), (cuuint64_t)tuples};
      const cuuint64_t strides[1] = {(cuuint64_t)(8u << K)};
      const cuuint32_t box[2] = {32, (cuuint32_t)kGtTuples};   // (32 floats, 32 rows)
      const cuuint32_t es[2] = {1, 1};
      rc = enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, base, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
               CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    } else {
      const uint64_t high = tuples >> q;
      if (high >= (1ull << 31) || q > 30) return false;
      const int ql = std::min(q, 5);
      const cuuint64_t dims[3] = {(cuuint64_t)(2ull << q), (cuuint64_t)(1u << K), (cuuint64_t)high};
      const cuuint64_t strides[2] = {(cuuint64_t)(8ull << q), (cuuint64_t)(8ull << (q + K))};
      const cuuint32_t box[3] = {(cuuint32_t)std::min(2 << ql, 64), (cuuint32_t)(1u << K), (cuuint32_t)(1u << (5 - ql))};
      const cuuint32_t es[3] = {1, 1, 1};
      rc = enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, base, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
               CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    }
    if (rc != CUDA_SUCCESS) return false;
  }
  return true;
}

template <int K>
static int launch_gram_tma(const float2* psi, const float2* lam, int n, int q, double* partials, int* grid_out,
                           cudaStream_t st, bool* done) {
  using L = GramTmaSmem<K>;
  *done = false;
  if (n - K < 5 || (n - K) >= 31 + 5) return QS_OK;
  CUtensorMap mp, ml;
  if (!gram_maps<K>(psi, lam, n, q, &mp, &ml)) return QS_OK;
  int dev = 0, sms = 0;
  QS_CUDA(cudaGetDevice(&dev));
  QS_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const uint64_t total = 1ull << (n - K);
  const uint64_t tiles = total / kGtTuples;
  const unsigned grid = (unsigned)std::min<uint64_t>(tiles, (uint64_t)sms);
  if (q == 0) {
    QS_CUDA(cudaFuncSetAttribute(k_gram_tma<K, TMA_ROWS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L::BYTES));
    k_gram_tma<K, TMA_ROWS><<<grid, kGtThreads, L::BYTES, st>>>(mp, ml, total, q, partials);
  } else {
    QS_CUDA(cudaFuncSetAttribute(k_gram_tma<K, TMA_MEMBERS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L::BYTES));
    k_gram_tma<K, TMA_MEMBERS><<<grid, kGtThreads, L::BYTES, st>>>(mp, ml, total, q, partials);
  }
  QS_LAUNCHED();
  *grid_out = (int)grid;
  *done = true;
  return QS_OK;
}

// Real Gram matrix of a 4- or 5-qubit support (qubits ascending) over a
// complex64 register, interleaved layout, partials [grid][W][W]; *grid_out
// receives the row count for the fold.
int gram_tc(int w, const float2* psi, const float2* lam, int n, const int* qubits, double* partials, int* grid_out,
            cudaStream_t st) {
  if (g_tma_enabled && (w == 4 || w == 5) && qubits[w - 1] == qubits[0] + w - 1) {
    bool done = false;
    if (w == 4) QS_TRY(launch_gram_tma<4>(psi, lam, n, qubits[0], partials, grid_out, st, &done));
    else QS_TRY(launch_gram_tma<5>(psi, lam, n, qubits[0], partials, grid_out, st, &done));
    if (done) return QS_OK;
  }
  if (w == 4) return launch_gram_tc_t<4>(psi, lam, n, qubits, partials, grid_out, st);
  if (w == 5) return launch_gram_tc_t<5>(psi, lam, n, qubits, partials, grid_out, st);
  return fail(QS_EUNSUPPORTED, "tensor-core Gram takes 4- or 5-qubit supports");
}

static int g_tc_enabled = 1;

void set_tensor_cores(int mode) { g_tc_enabled = mode < 0 ? 0 : (mode > 2 ? 2 : mode); }
int tensor_cores_enabled() { return g_tc_enabled; }

// 0: never; 2: always (complex64 dense k = 4, 5); 1 (default): where the
// tensor-core kernel measured faster than the CUDA-core one on GB300 at n = 25:
// k = 5 unless qubit 0 is free and no target is below qubit 5 (those tuples are
// gathered with fully coalesced pairs by the CUDA-core kernel), and k = 4 when
// qubit 0 is a target.
bool use_block_tc(int dtype, const Plan& p) {
  if (!g_tc_enabled || dtype != QS_C64 || p.op != OP_DENSEK || (p.k != 4 && p.k != 5)) return false;
  if (g_tc_enabled == 2) return true;
  int lo = 64;
  bool q0 = false;
  for (int j = 0; j < p.k; ++j) {
    lo = std::min(lo, p.locs[j]);
    q0 = q0 || p.locs[j] == 0;
  }
  // consecutive targets without controls take the TMA-fed kernel, faster than
  // the CUDA-core kernel at every such placement measured (k = 4 and 5)
  int hi = 0;
  for (int j = 0; j < p.k; ++j) hi = std::max(hi, p.locs[j]);
  if (g_tma_enabled && p.ctrl_mask == 0 && hi - lo == p.k - 1) return true;
  if (p.k == 4) return q0;
  return q0 || lo < 5 || (p.ctrl_mask & 1ull);
}

int launch_block_tc(float2* psi, int n, int nreg, const Plan& p, cudaStream_t st) {
  if (p.k == 4) return launch_tc_t<4>(psi, n, nreg, p, st);
  if (p.k == 5) return launch_tc_t<5>(psi, n, nreg, p, st);
  return fail(QS_EUNSUPPORTED, "tensor-core blocks take 4 or 5 targets");
}

// device address of the status word on the current device, for kernels of
// other files that report a bounded wait that gave up
int tc_status_address(int** out) {
  void* p = nullptr;
  QS_CUDA(cudaGetSymbolAddress(&p, g_tc_status));
  *out = (int*)p;
  return QS_OK;
}

// reads and clears the device status word (synchronous)
int tc_status_take() {
  int e = 0;
  QS_CUDA(cudaMemcpyFromSymbol(&e, g_tc_status, sizeof(int)));
  if (e) {
    const int z = 0;
    QS_CUDA(cudaMemcpyToSymbol(g_tc_status, &z, sizeof(int)));
    return fail(QS_ETIMEDOUT, "a bounded device-side wait (tensor-core pipeline or grid barrier) gave up");
  }
  return QS_OK;
}

// One thread waits on an mbarrier whose phase nothing completes, through the
// same bounded wait as the tensor-core pipeline, and reports through the same
// device status word.
__global__ void k_wait_selftest(uint64_t limit_ns, int* out) {
  __shared__ __align__(8) uint64_t bar;
  __shared__ int abort_flag;
  const uint32_t mb = smem_u32(&bar);
  mbar_init(mb, 1);
  abort_flag = 0;
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  const uint64_t t0 = global_ns();
  const bool ok = mbar_wait(mb, 0, &abort_flag, limit_ns);
  const uint64_t t1 = global_ns();
  if (!ok) atomicExch(&g_tc_status, 1);
  out[0] = ok ? 1 : 0;
  out[1] = abort_flag;
  out[2] = (int)((t1 - t0) / 1000ull);  // microseconds waited
}

}  // namespace qs

using namespace qs;

extern "C" int qs_selftest_bounded_wait(double limit_ms, int* host_result) {
  if (!host_result || !(limit_ms > 0) || limit_ms > 1000) return fail(QS_EINVAL, "limit_ms must be in (0, 1000]");
  int* d = nullptr;
  QS_CUDA(cudaMalloc(&d, 3 * sizeof(int)));
  k_wait_selftest<<<1, 1>>>((uint64_t)(limit_ms * 1e6), d);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpy(host_result, d, 3 * sizeof(int), cudaMemcpyDeviceToHost);
  cudaFree(d);
  if (e != cudaSuccess) return fail(QS_EDEVICE, "wait self-test: %s", cudaGetErrorString(e));
  return tc_status_take();
}
