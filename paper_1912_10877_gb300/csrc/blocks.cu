// blocks.cu -- fusion of a circuit's gates into k-qubit blocks (k <= 5) and
// the autotuner that picks the fusion width or the tile shape for a circuit.
//
// Sec. "Performance" applies every gate through the general multi-qubit
// instruction; a chain of gates acting on at most k qubits is itself one such
// instruction with the product matrix (Sec. "Matrix Representation": the
// matrix of a chain is the product of its blocks' matrices).  Fusing adjacent
// gates into blocks trades HBM passes (one per block instead of one per gate)
// for arithmetic per amplitude (2^k complex multiply-adds), and dense blocks
// of 4 and 5 qubits run on the tensor cores.
//
// The reversible backward over blocks (Sec. "Reverse Mode" with blocks as the
// unit): walking the blocks from last to first with psi and lambda the states
// right after block B = G_m ... G_1 (support S, 2^w = D), every gate G_j of B
// with a parameter has psi_j = E_j^dag psi, lambda_j = E_j^dag lambda, where
// E_j = G_m ... G_{j+1} acts on S only.  So
//   <lambda_j|H_j|psi_j> = Tr(E_j H_j E_j^dag rho),  rho = sum_x psi_x lambda_x^dag,
// the sum running over the 2^(n-w) tuples x of S.  One pass over psi and
// lambda forms the D x D matrix rho; every gradient of the block then follows
// on the host in FP64, and both states are uncomputed by B^dag.
//
// The planner walks the gates in order and keeps several open blocks with
// pairwise disjoint supports (so they commute).  A gate joins the open blocks
// it touches when the union of their supports and its own qubits (targets and
// controls) has at most k qubits; otherwise those blocks are emitted and the
// gate opens a new one.  The structure depends only on the gate list; the
// matrices are formed for each parameter vector.
#include <chrono>
#include <cstring>
#include <type_traits>

#include "common.cuh"

namespace qs {

namespace {

struct Block {
  uint64_t support = 0;      // register qubits (targets and controls of its gates)
  std::vector<int> gates;    // circuit gate indices in application order
};

int popc(uint64_t m) { return __builtin_popcountll(m); }

uint64_t gate_qubits(const qs_gate_desc& g) {
  uint64_t m = g.ctrl_mask;
  for (int j = 0; j < g.nlocs; ++j) m |= 1ull << g.locs[j];
  return m;
}

void plan_blocks(const qs_circuit* c, int kmax, std::vector<Block>& out) {
  out.clear();
  std::vector<Block> open;
  for (int gi = 0; gi < (int)c->gates.size(); ++gi) {
    const uint64_t q = gate_qubits(c->gates[gi]);
    uint64_t s = q;
    for (const Block& b : open)
      if (b.support & q) s |= b.support;
    if (popc(s) <= kmax) {
      Block merged;
      merged.support = s;
      std::vector<Block> rest;
      for (Block& b : open) {
        if (b.support & q) merged.gates.insert(merged.gates.end(), b.gates.begin(), b.gates.end());
        else rest.push_back(std::move(b));
      }
      merged.gates.push_back(gi);
      rest.push_back(std::move(merged));
      open.swap(rest);
      continue;
    }
    // The union is too wide.  Keep the widest touched block that can still take
    // the gate open and close the other touched blocks (open blocks are
    // disjoint, so the closed ones commute with it and may be applied first);
    // if none can take it, close them all and start a block with the gate.
    long keep = -1;
    for (size_t i = 0; i < open.size(); ++i)
      if ((open[i].support & q) && popc(open[i].support | q) <= kmax &&
          (keep < 0 || popc(open[i].support) > popc(open[(size_t)keep].support)))
        keep = (long)i;
    std::vector<Block> rest;
    for (size_t i = 0; i < open.size(); ++i) {
      Block& b = open[i];
      if ((long)i == keep) continue;
      if (b.support & q) out.push_back(std::move(b));
      else rest.push_back(std::move(b));
    }
    if (keep >= 0) {
      Block kb = std::move(open[(size_t)keep]);
      kb.support |= q;
      kb.gates.push_back(gi);
      rest.push_back(std::move(kb));
    } else {
      Block nb;
      nb.support = q;
      nb.gates.push_back(gi);
      if (popc(q) > kmax) out.push_back(std::move(nb));  // wider than k: stays a gate of its own
      else rest.push_back(std::move(nb));
    }
    open.swap(rest);
  }
  for (Block& b : open) out.push_back(std::move(b));
  // Commutation-aware merging: block j may move earlier past blocks whose
  // support is disjoint from its own (they commute), so it joins the earliest
  // block it can reach whose union with it still spans at most kmax qubits
  // (the nearest earlier block that shares a qubit with j ends the search).
  // The greedy pass above closes every open block a gate touches when their
  // union is too wide, which leaves many 1-3-qubit blocks; each costs a full
  // pass over the state, as much as a 5-qubit block.
  // Then the mirror image: block i may move later past disjoint blocks and join
  // the latest block it can reach (its gates go first in the merged block).
  bool changed = true;
  while (changed) {
    changed = false;
    for (size_t j = 1; j < out.size();) {
      const uint64_t sj = out[j].support;
      long best = -1;
      if (popc(sj) <= kmax) {
        for (long i = (long)j - 1; i >= 0; --i) {
          const uint64_t si = out[(size_t)i].support;
          if (popc(si | sj) <= kmax) {
            best = i;
            if (si & sj) break;
          } else if (si & sj) {
            break;
          }
        }
      }
      if (best >= 0) {
        Block& t = out[(size_t)best];
        t.support |= sj;
        t.gates.insert(t.gates.end(), out[j].gates.begin(), out[j].gates.end());
        out.erase(out.begin() + (long)j);
        changed = true;
      } else {
        ++j;
      }
    }
    for (long i = (long)out.size() - 2; i >= 0; --i) {
      const uint64_t si = out[(size_t)i].support;
      if (popc(si) > kmax) continue;
      long best = -1;
      for (size_t j = (size_t)i + 1; j < out.size(); ++j) {
        const uint64_t sj = out[j].support;
        if (popc(si | sj) <= kmax) {
          best = (long)j;
          if (si & sj) break;
        } else if (si & sj) {
          break;
        }
      }
      if (best >= 0) {
        Block& t = out[(size_t)best];
        t.support |= si;
        t.gates.insert(t.gates.begin(), out[(size_t)i].gates.begin(), out[(size_t)i].gates.end());
        out.erase(out.begin() + i);
        changed = true;
      }
    }
  }
}

// M <- G M for a gate G (matrix U over targets tpos, controls cmask/cval) on
// the w-qubit block space; M is 2^w x 2^w row-major
void left_multiply(std::vector<cd>& M, int w, const std::vector<cd>& U, int k, const int* tpos, uint32_t cmask,
                   uint32_t cval) {
  const int Dw = 1 << w, Dk = 1 << k;
  uint32_t tmask = 0;
  std::vector<uint32_t> off(Dk, 0);
  for (int j = 0; j < k; ++j) tmask |= 1u << tpos[j];
  for (int m = 0; m < Dk; ++m)
    for (int j = 0; j < k; ++j)
      if ((m >> j) & 1) off[m] |= 1u << tpos[j];
  std::vector<cd> v(Dk);
  for (int col = 0; col < Dw; ++col)
    for (uint32_t x = 0; x < (uint32_t)Dw; ++x) {
      if ((x & tmask) || (x & cmask) != cval) continue;
      for (int m = 0; m < Dk; ++m) v[m] = M[(size_t)(x | off[m]) * Dw + col];
      for (int r = 0; r < Dk; ++r) {
        cd acc = 0;
        for (int m = 0; m < Dk; ++m) acc += U[(size_t)r * Dk + m] * v[m];
        M[(size_t)(x | off[r]) * Dw + col] = acc;
      }
    }
}

// the block's qubits (ascending) and its 2^w x 2^w matrix (bit j <-> qubits[j])
int block_matrix(const qs_circuit* c, const Block& b, const double* params, std::vector<int>& qubits,
                 std::vector<cd>& M) {
  qubits.clear();
  for (int q = 0; q < 64; ++q)
    if ((b.support >> q) & 1ull) qubits.push_back(q);
  const int w = (int)qubits.size();
  int pos[64];
  for (int j = 0; j < w; ++j) pos[qubits[j]] = j;
  M.assign((size_t)1 << (2 * w), cd(0));
  for (int i = 0; i < (1 << w); ++i) M[(size_t)i * (1 << w) + i] = 1;
  std::vector<cd> U;
  for (int gi : b.gates) {
    const qs_gate_desc& g = c->gates[gi];
    QS_TRY(gate_matrix(c, g, params, U));
    int tpos[QS_MAXK];
    for (int j = 0; j < g.nlocs; ++j) tpos[j] = pos[g.locs[j]];
    uint32_t cmask = 0, cval = 0;
    for (int q = 0; q < 64; ++q)
      if ((g.ctrl_mask >> q) & 1ull) {
        cmask |= 1u << pos[q];
        if ((g.ctrl_vals >> q) & 1ull) cval |= 1u << pos[q];
      }
    left_multiply(M, w, U, g.nlocs, tpos, cmask, cval);
  }
  return QS_OK;
}

const std::vector<Block>& cached_blocks(const qs_circuit* c, int kmax) {
  if (c->block_k != kmax || !c->blocks) {
    auto* v = new std::vector<Block>();
    plan_blocks(c, kmax, *v);
    delete static_cast<std::vector<Block>*>(c->blocks);
    c->blocks = v;
    c->block_k = kmax;
  }
  return *static_cast<const std::vector<Block>*>(c->blocks);
}

}  // namespace

void free_blocks(const qs_circuit* c) {
  delete static_cast<std::vector<Block>*>(c->blocks);
  c->blocks = nullptr;
}

int apply_blocks(qs_state* s, const qs_circuit* c, const double* params, int kmax, bool precise) {
  if (kmax < 1 || kmax > QS_MAXK) return fail(QS_EINVAL, "block width %d not in 1..%d", kmax, QS_MAXK);
  const std::vector<Block>& blocks = cached_blocks(c, kmax);
  std::vector<int> qubits;
  std::vector<cd> M;
  for (const Block& b : blocks) {
    Plan p;
    if (b.gates.size() == 1) {  // a lone gate keeps its controls as controls
      const qs_gate_desc& g = c->gates[b.gates[0]];
      QS_TRY(gate_matrix(c, g, params, M));
      QS_TRY(plan_gate(M.data(), g.nlocs, g.locs, g.ctrl_mask, g.ctrl_vals, &p));
    } else {
      QS_TRY(block_matrix(c, b, params, qubits, M));
      QS_TRY(plan_gate(M.data(), (int)qubits.size(), qubits.data(), 0, 0, &p));
    }
    p.precise = precise && s->dtype == QS_C64;
    QS_TRY(launch_plan(s, p));
  }
  return QS_OK;
}

// ------------------------------------------------------------------ block backward

namespace {

constexpr int kGramThreads = 256;
constexpr int kGramRows = 128;  // tuples staged per tile

template <int D>
struct GramArgs {
  uint64_t total;             // tuples
  uint64_t reg_stride;
  IdxSpec s;                  // tuple base index (support bits fixed at 0)
  int lowbits;                // support qubits 0..lowbits-1 are register qubits 0..lowbits-1
  uint32_t off[D];            // member offsets (support qubits ascending)
};

template <typename R> struct AmpOf;
template <> struct AmpOf<float> { using T = float2; };
template <> struct AmpOf<double> { using T = double2; };

// Per-CTA FP64 partials of the real Gram matrix G = A^T B over all tuples,
// A = [Re psi_x | Im psi_x], B = [Re lambda_x | Im lambda_x] (rows = tuples).
// Thread layout: the (2D)^2 entries are split into RB x RB sub-blocks, one
// per thread of a group; groups split the tuples of a tile.  Products are
// summed in R over a tile, then added to FP64 accumulators.
template <typename R, int D>
__global__ void __launch_bounds__(kGramThreads) k_gram(const typename AmpOf<R>::T* __restrict__ psi,
                                                       const typename AmpOf<R>::T* __restrict__ lam,
                                                       const __grid_constant__ GramArgs<D> a,
                                                       double* __restrict__ partials) {
  constexpr int W2 = 2 * D, E = W2 * W2;
  constexpr int EPT = E >= 16 * kGramThreads ? 16 : (E >= 4 * kGramThreads ? 4 : 1);
  constexpr int RB = EPT == 16 ? 4 : (EPT == 4 ? 2 : 1);
  constexpr int NTG = E / EPT;                 // threads covering all entries once
  constexpr int G = kGramThreads / NTG;        // groups
  static_assert(NTG * G == kGramThreads && NTG * EPT == E, "thread layout");
  extern __shared__ unsigned char gsm[];
  R* As = reinterpret_cast<R*>(gsm);                        // [kGramRows][W2]
  R* Bs = As + kGramRows * W2;                              // [kGramRows][W2]
  uint64_t* sb = reinterpret_cast<uint64_t*>(Bs + kGramRows * W2);
  uint32_t* soff = reinterpret_cast<uint32_t*>(sb + kGramRows);
  const int tid = threadIdx.x, grp = tid / NTG, li = tid % NTG;
  if (tid < D) soff[tid] = a.off[tid];
  const int r0 = (li / (W2 / RB)) * RB, c0 = (li % (W2 / RB)) * RB;
  const int lb = a.lowbits;
  const uint32_t lowmask = (1u << lb) - 1u;
  // element (t, col) of a tile row lives at t W2 + swizzled 16-byte chunk: the
  // chunk index is XORed with t, so that writes of one column by consecutive
  // rows and 16-byte reads of one row both spread over the banks
  constexpr int CM = W2 >= 8 ? W2 / 4 - 1 : 0;
  auto sw = [](int t, int col) { return t * W2 + ((((col >> 2) ^ (t & CM)) & CM) << 2) + (col & 3) + (CM ? 0 : (col & ~3)); };
  double accd[RB][RB];
#pragma unroll
  for (int i = 0; i < RB; ++i)
#pragma unroll
    for (int j = 0; j < RB; ++j) accd[i][j] = 0.0;
  for (uint64_t t0 = (uint64_t)blockIdx.x * kGramRows; t0 < a.total; t0 += (uint64_t)gridDim.x * kGramRows) {
    const int rows = a.total - t0 < (uint64_t)kGramRows ? (int)(a.total - t0) : kGramRows;
    if (tid < kGramRows) {
      const uint64_t t = t0 + tid;
      uint64_t b = 0;
      if (t < a.total) {
        const uint64_t r = t >> a.s.item_log2, j = t & ((1ull << a.s.item_log2) - 1ull);
        b = r * a.reg_stride + deposit(j, a.s);
      }
      sb[tid] = b;
    }
    __syncthreads();
    for (int e = tid; e < kGramRows * D; e += kGramThreads) {
      const int t = (e >> lb) & (kGramRows - 1);
      const int m = (int)(((uint32_t)e & lowmask) | (((uint32_t)e >> (lb + 7)) << lb));
      typename AmpOf<R>::T x{}, y{};
      if (t < rows) {
        const uint64_t idx = sb[t] + soff[m];
        x = psi[idx];
        y = lam[idx];
      }
      As[sw(t, m)] = x.x;
      As[sw(t, D + m)] = x.y;
      Bs[sw(t, m)] = y.x;
      Bs[sw(t, D + m)] = y.y;
    }
    __syncthreads();
    R acc[RB][RB];
#pragma unroll
    for (int i = 0; i < RB; ++i)
#pragma unroll
      for (int j = 0; j < RB; ++j) acc[i][j] = 0;
    for (int t = grp; t < rows; t += G) {
      R av[RB], bv[RB];
      if constexpr (RB == 4 && sizeof(R) == 4) {  // one 16-byte load per operand
        const float4 x = *reinterpret_cast<const float4*>(As + sw(t, r0));
        const float4 y = *reinterpret_cast<const float4*>(Bs + sw(t, c0));
        av[0] = x.x; av[1] = x.y; av[2] = x.z; av[3] = x.w;
        bv[0] = y.x; bv[1] = y.y; bv[2] = y.z; bv[3] = y.w;
      } else {
#pragma unroll
        for (int i = 0; i < RB; ++i) {
          av[i] = As[sw(t, r0 + i)];
          bv[i] = Bs[sw(t, c0 + i)];
        }
      }
#pragma unroll
      for (int i = 0; i < RB; ++i)
#pragma unroll
        for (int j = 0; j < RB; ++j) acc[i][j] = fma(av[i], bv[j], acc[i][j]);
    }
#pragma unroll
    for (int i = 0; i < RB; ++i)
#pragma unroll
      for (int j = 0; j < RB; ++j) accd[i][j] += (double)acc[i][j];
    __syncthreads();
  }
  double* out = partials + (size_t)blockIdx.x * E;
  if constexpr (G == 1) {
#pragma unroll
    for (int i = 0; i < RB; ++i)
#pragma unroll
      for (int j = 0; j < RB; ++j) out[(r0 + i) * W2 + c0 + j] = accd[i][j];
  } else {
    // groups summed in group order (G * E = 256 doubles fit in the operand tiles)
    static_assert(G * E * sizeof(double) <= 2 * kGramRows * W2 * sizeof(R), "group reduction fits");
    double* red = reinterpret_cast<double*>(gsm);
    red[grp * E + r0 * W2 + c0] = accd[0][0];
    __syncthreads();
    for (int e = tid; e < E; e += kGramThreads) {
      double acc = 0.0;
      for (int g = 0; g < G; ++g) acc += red[g * E + e];
      out[e] = acc;
    }
  }
}

// The same partials for complex64 supports of 1..3 qubits without staging:
// each warp walks whole 128-tuple tiles; a group of SPLIT lanes shares one
// tuple (lane j of the group takes psi rows [j RPL, (j+1) RPL) of the 2D
// rows (member, re/im) and every lambda member), so a lane keeps RPL x 2D FP32
// products of its tuples in registers (16 or 32).  Each iteration loads two
// tuple steps before multiplying, so two steps of loads are in flight per
// warp.  Every 16 steps the lanes of a warp fold their FP32 sums with
// shuffles (fixed tree) and add them to per-warp FP64 accumulators in shared
// memory; the warps are added in warp order at the end.
template <int D>
__global__ void __launch_bounds__(256, 3) k_gram_reg(const float2* __restrict__ psi, const float2* __restrict__ lam,
                                                     const __grid_constant__ GramArgs<D> a, double* __restrict__ partials) {
  static_assert(D == 2 || D == 4 || D == 8, "1..3-qubit supports");
  constexpr int W2 = 2 * D, E = W2 * W2;
  constexpr int SPLIT = D == 2 ? 1 : (D == 4 ? 2 : 8);   // lanes per tuple
  constexpr int RPL = W2 / SPLIT;                  // psi rows per lane: 4, 4, 2
  constexpr int MPL = (RPL + 1) / 2;               // psi members loaded per lane
  constexpr int NACC = RPL * W2;                   // 16 / 32 / 32
  constexpr int TPW = 32 / SPLIT;                  // tuples per warp step
  constexpr int STEPS = kGramRows / TPW;           // steps per tile (even)
  constexpr int UNR = 2;                           // steps loaded together
  constexpr int FLUSH = 16;                        // steps between FP64 folds
  constexpr int NW = 256 / 32;
  static_assert(STEPS % UNR == 0 && FLUSH % UNR == 0, "step unrolling");
  extern __shared__ __align__(16) unsigned char gsm_reg[];
  double* wacc = reinterpret_cast<double*>(gsm_reg);                       // [NW][E]
  uint64_t* sP = reinterpret_cast<uint64_t*>(wacc + NW * E);                // [kGramRows]
  uint32_t* soff = reinterpret_cast<uint32_t*>(sP + kGramRows);             // [D]
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int j = lane % SPLIT, tup = lane / SPLIT;
  const int m0 = (j * RPL) >> 1;                   // first psi member of this lane
  for (int e = tid; e < NW * E; e += 256) wacc[e] = 0.0;
  if (tid < D) soff[tid] = a.off[tid];
  if (tid < kGramRows) {
    // offset of tile-local tuple t: deposit of t into the free bits (support bits zero)
    sP[tid] = deposit((uint64_t)tid & ((1ull << (a.s.item_log2 < 7 ? a.s.item_log2 : 7)) - 1ull), a.s) & ~a.s.set_bits;
  }
  __syncthreads();
  float acc[NACC];
#pragma unroll
  for (int e = 0; e < NACC; ++e) acc[e] = 0.f;
  int since = 0;
  auto flush = [&]() {
#pragma unroll
    for (int e = 0; e < NACC; ++e) {
      float v = acc[e];
#pragma unroll
      for (int o = SPLIT; o < 32; o <<= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      acc[e] = 0.f;
      if (tup == 0) wacc[warp * E + (j * RPL + e / W2) * W2 + e % W2] += (double)v;
    }
    since = 0;
  };
  const uint64_t ntiles = (a.total + kGramRows - 1) / kGramRows;
  const uint64_t per_reg = 1ull << a.s.item_log2;
  for (uint64_t tile = (uint64_t)blockIdx.x * NW + warp; tile < ntiles; tile += (uint64_t)gridDim.x * NW) {
    const uint64_t t0 = tile * kGramRows;
    const int rows = a.total - t0 < (uint64_t)kGramRows ? (int)(a.total - t0) : kGramRows;
    const uint64_t r = t0 / per_reg, jj = t0 % per_reg;
    const uint64_t tb = r * a.reg_stride + deposit(jj, a.s);
    for (int st = 0; st < STEPS; st += UNR) {
      float2 pv[UNR][MPL], lv[UNR][D];
#pragma unroll
      for (int u = 0; u < UNR; ++u) {
        const int t = (st + u) * TPW + tup;
        const bool ok = t < rows;
        const uint64_t base = tb + sP[ok ? t : 0];
#pragma unroll
        for (int m = 0; m < MPL; ++m) pv[u][m] = ok ? psi[base + soff[m0 + m]] : make_float2(0.f, 0.f);
#pragma unroll
        for (int m = 0; m < D; ++m) lv[u][m] = ok ? lam[base + soff[m]] : make_float2(0.f, 0.f);
      }
#pragma unroll
      for (int u = 0; u < UNR; ++u) {
#pragma unroll
        for (int rr = 0; rr < RPL; ++rr) {
          // local row rr is 2D row j RPL + rr: member (j RPL + rr) / 2, re (even) or im (odd)
          const float v = (((j * RPL + rr) & 1) == 0) ? pv[u][rr >> 1].x : pv[u][rr >> 1].y;
#pragma unroll
          for (int c = 0; c < D; ++c) {
            acc[rr * W2 + c] = fmaf(v, lv[u][c].x, acc[rr * W2 + c]);
            acc[rr * W2 + D + c] = fmaf(v, lv[u][c].y, acc[rr * W2 + D + c]);
          }
        }
      }
      since += UNR;
      if (since == FLUSH) flush();
    }
  }
  flush();
  __syncthreads();
  // rows of this layout are (member, re/im) pairs; the partials use rows m (re) and D + m (im)
  for (int e = tid; e < E; e += 256) {
    const int r = e / W2, c = e % W2;
    const int m = r >> 1, part = r & 1;
    double v = 0.0;
    for (int w = 0; w < NW; ++w) v += wacc[w * E + e];
    partials[(size_t)blockIdx.x * E + (part * D + m) * W2 + c] = v;
  }
}

template <int D>
constexpr size_t gram_reg_smem() { return sizeof(double) * 8 * (2 * D) * (2 * D) + 8 * kGramRows + 4 * D; }

// out[e] = sum over rows of partials[row][e]: one CTA per entry, rows strided
// over the threads, then a fixed-shape tree (the result does not depend on timing)
__global__ void __launch_bounds__(256) k_gram_fold(const double* __restrict__ partials, int nrows, int E,
                                                   double* __restrict__ out) {
  __shared__ double red[256];
  const int e = blockIdx.x;
  double acc = 0.0;
  for (int r = threadIdx.x; r < nrows; r += 256) acc += partials[(size_t)r * E + e];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int h = 128; h > 0; h >>= 1) {
    if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[e] = red[0];
}

// lambda (+)= O psi for one register, terms in chunks (Pauli strings X^x Z^z with i^{popcount(x&z)})
constexpr int kObsTerms = 32;
struct ObsTerms {
  int nt;
  uint64_t x[kObsTerms], z[kObsTerms];
  int ny[kObsTerms];
  double c[kObsTerms];
};

template <typename R>
__global__ void __launch_bounds__(256) k_obs(const typename AmpOf<R>::T* __restrict__ psi,
                                             typename AmpOf<R>::T* __restrict__ lam, uint64_t dim, int accumulate,
                                             const __grid_constant__ ObsTerms o) {
  const uint64_t i = (uint64_t)blockIdx.x * 256 + threadIdx.x;
  if (i >= dim) return;
  typename AmpOf<R>::T acc = accumulate ? lam[i] : typename AmpOf<R>::T{};
  for (int t = 0; t < o.nt; ++t) {
    const uint64_t j = i ^ o.x[t];
    const typename AmpOf<R>::T v = psi[j];
    const R sgn = (R)((__popcll(j & o.z[t]) & 1) ? -o.c[t] : o.c[t]);
    R re, im;
    switch (o.ny[t] & 3) {
      case 0: re = v.x; im = v.y; break;
      case 1: re = -v.y; im = v.x; break;
      case 2: re = -v.x; im = -v.y; break;
      default: re = v.y; im = -v.x; break;
    }
    acc.x = fma(sgn, re, acc.x);
    acc.y = fma(sgn, im, acc.y);
  }
  lam[i] = acc;
}

template <typename R>
int apply_obs(const void* psi, void* lam, int n, const qs_observable* o, cudaStream_t st) {
  using T = typename AmpOf<R>::T;
  const uint64_t dim = 1ull << n;
  const int nt = (int)o->terms.size();
  if (nt == 0) {
    QS_CUDA(cudaMemsetAsync(lam, 0, sizeof(T) * dim, st));
    return QS_OK;
  }
  for (int c0 = 0; c0 < nt; c0 += kObsTerms) {
    ObsTerms ch;
    std::memset(&ch, 0, sizeof(ch));
    ch.nt = std::min(kObsTerms, nt - c0);
    for (int t = 0; t < ch.nt; ++t) {
      const qs_pauli_term& term = o->terms[c0 + t];
      ch.x[t] = term.x_mask;
      ch.z[t] = term.z_mask;
      ch.ny[t] = popc(term.x_mask & term.z_mask) & 3;
      ch.c[t] = term.coeff;
    }
    k_obs<R><<<(unsigned)((dim + 255) / 256), 256, 0, st>>>((const T*)psi, (T*)lam, dim, c0 > 0, ch);
    QS_LAUNCHED();
  }
  return QS_OK;
}

template <typename R, int D>
int launch_gram(const void* psi, const void* lam, int n, const std::vector<int>& qubits, double* partials,
                double* folded, cudaStream_t st) {
  constexpr int W2 = 2 * D, E = W2 * W2;
  GramArgs<D> a;
  std::memset(&a, 0, sizeof(a));
  uint64_t mask = 0;
  for (int q : qubits) mask |= 1ull << q;
  QS_TRY(make_idx(n, mask, 0, &a.s));
  a.reg_stride = 1ull << n;
  a.total = 1ull << a.s.item_log2;
  a.lowbits = 0;
  while (a.lowbits < (int)qubits.size() && qubits[a.lowbits] == a.lowbits) ++a.lowbits;
  for (int m = 0; m < D; ++m) {
    uint64_t o = 0;
    for (int j = 0; j < (int)qubits.size(); ++j)
      if ((m >> j) & 1) o |= 1ull << qubits[j];
    a.off[m] = (uint32_t)o;
  }
  int dev = 0, sms = 0, per_sm = 0;
  QS_CUDA(cudaGetDevice(&dev));
  if constexpr (std::is_same<R, float>::value && (D == 2 || D == 4 || D == 8)) {
    constexpr size_t rsm = gram_reg_smem<D>();
    QS_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    QS_CUDA(cudaFuncSetAttribute(k_gram_reg<D>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rsm));
    QS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_gram_reg<D>, 256, rsm));
    if (per_sm < 1) return fail(QS_EDEVICE, "Gram kernel does not fit on an SM");
    const uint64_t tiles = (a.total + kGramRows - 1) / kGramRows;
    const int grid = (int)std::max<uint64_t>(1, std::min<uint64_t>((tiles + 7) / 8, (uint64_t)sms * per_sm));
    k_gram_reg<D><<<grid, 256, rsm, st>>>((const float2*)psi, (const float2*)lam, a, partials);
    QS_LAUNCHED();
    k_gram_fold<<<E, 256, 0, st>>>(partials, grid, E, folded);
    QS_LAUNCHED();
    return QS_OK;
  }
  const size_t smem = 2 * (size_t)kGramRows * W2 * sizeof(R) + kGramRows * 8 + D * 4;
  QS_CUDA(cudaFuncSetAttribute(k_gram<R, D>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  QS_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  QS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_gram<R, D>, kGramThreads, smem));
  if (per_sm < 1) return fail(QS_EDEVICE, "Gram kernel does not fit on an SM");
  const uint64_t tiles = (a.total + kGramRows - 1) / kGramRows;
  const int grid = (int)std::min<uint64_t>(tiles, (uint64_t)sms * per_sm);
  k_gram<R, D><<<grid, kGramThreads, smem, st>>>((const typename AmpOf<R>::T*)psi,
                                                  (const typename AmpOf<R>::T*)lam, a, partials);
  QS_LAUNCHED();
  k_gram_fold<<<E, 256, 0, st>>>(partials, grid, E, folded);
  QS_LAUNCHED();
  return QS_OK;
}

// rows x entries of the partials for a block of width w (upper bound over the grid)
size_t gram_partials_doubles(int sms) {
  size_t best = 0;
  for (int w = 0; w <= QS_MAXK; ++w) {
    const size_t W2 = (size_t)2 << w, E = W2 * W2;
    const size_t ept = E >= 16 * kGramThreads ? 16 : (E >= 4 * kGramThreads ? 4 : 1);
    (void)ept;
    best = std::max(best, (size_t)sms * 8 * E);
  }
  return best;
}

template <typename R>
int gram(int w, const void* psi, const void* lam, int n, const std::vector<int>& qubits, double* partials,
         double* folded, cudaStream_t st) {
  switch (w) {
    case 0: return launch_gram<R, 1>(psi, lam, n, qubits, partials, folded, st);
    case 1: return launch_gram<R, 2>(psi, lam, n, qubits, partials, folded, st);
    case 2: return launch_gram<R, 4>(psi, lam, n, qubits, partials, folded, st);
    case 3: return launch_gram<R, 8>(psi, lam, n, qubits, partials, folded, st);
    case 4: return launch_gram<R, 16>(psi, lam, n, qubits, partials, folded, st);
    case 5: return launch_gram<R, 32>(psi, lam, n, qubits, partials, folded, st);
  }
  return fail(QS_EUNSUPPORTED, "block of %d qubits", w);
}

// H embedded in the block space: acts as H on the targets where the controls
// match, and as zero elsewhere (the control projector)
void embed_generator(const std::vector<cd>& H, int k, const int* tpos, uint32_t cmask, uint32_t cval, int w,
                     std::vector<cd>& out) {
  const int Dw = 1 << w, Dk = 1 << k;
  out.assign((size_t)Dw * Dw, cd(0));
  uint32_t tmask = 0;
  std::vector<uint32_t> off(Dk, 0);
  for (int j = 0; j < k; ++j) tmask |= 1u << tpos[j];
  for (int m = 0; m < Dk; ++m)
    for (int j = 0; j < k; ++j)
      if ((m >> j) & 1) off[m] |= 1u << tpos[j];
  for (uint32_t x = 0; x < (uint32_t)Dw; ++x) {
    if ((x & tmask) || (x & cmask) != cval) continue;
    for (int r = 0; r < Dk; ++r)
      for (int c = 0; c < Dk; ++c) out[(size_t)(x | off[r]) * Dw + (x | off[c])] = H[(size_t)r * Dk + c];
  }
}

// rho <- G^dag rho G for a gate G on the block space (both sides, O(D^2 2^k))
void conj_by_gate(std::vector<cd>& rho, int w, const std::vector<cd>& U, int k, const int* tpos, uint32_t cmask,
                  uint32_t cval) {
  const int D = 1 << w, Dk = 1 << k;
  std::vector<cd> Ud((size_t)Dk * Dk);
  for (int r = 0; r < Dk; ++r)
    for (int c = 0; c < Dk; ++c) Ud[(size_t)r * Dk + c] = std::conj(U[(size_t)c * Dk + r]);
  left_multiply(rho, w, Ud, k, tpos, cmask, cval);  // G^dag rho
  std::vector<cd> t((size_t)D * D);                 // (G^dag rho) G = (G^dag (G^dag rho)^dag)^dag
  for (int i = 0; i < D; ++i)
    for (int j = 0; j < D; ++j) t[(size_t)i * D + j] = std::conj(rho[(size_t)j * D + i]);
  left_multiply(t, w, Ud, k, tpos, cmask, cval);
  for (int i = 0; i < D; ++i)
    for (int j = 0; j < D; ++j) rho[(size_t)i * D + j] = std::conj(t[(size_t)j * D + i]);
}

}  // namespace

int backward_blocks(qs_state* s, const qs_circuit* c, const double* params, const qs_observable* o, int kmax,
                    void* work, double* host_grad, double* host_loss) {
  if (s->nreg != 1) return fail(QS_EUNSUPPORTED, "the block backward takes a single register");
  const int n = s->nq[0];
  if (n != c->nqubits) return fail(QS_EINVAL, "circuit has %d qubits, state %d", c->nqubits, n);
  if (kmax < 1 || kmax > QS_MAXK) return fail(QS_EINVAL, "block width %d not in 1..%d", kmax, QS_MAXK);
  if (!work || !host_grad) return fail(QS_EINVAL, "null argument");
  if (c->nparams > 0 && !params) return fail(QS_EINVAL, "params is NULL");
  const std::vector<Block>& blocks = cached_blocks(c, kmax);
  const int nb = (int)blocks.size();
  // which blocks need rho, and where it goes in device scratch
  std::vector<int64_t> rho_off(nb, -1);
  std::vector<char> rho_tc(nb, 0);  // rho of this block came from the tensor cores (interleaved layout)
  int64_t rho_total = 0;
  for (int bi = 0; bi < nb; ++bi) {
    const Block& b = blocks[bi];
    if (popc(b.support) > QS_MAXK) return fail(QS_EUNSUPPORTED, "a gate acts on more than %d qubits", QS_MAXK);
    bool has_param = false;
    for (int gi : b.gates) has_param = has_param || (c->gates[gi].param >= 0 && c->gates[gi].kind != QS_GATE_MATRIX);
    if (has_param) {
      rho_off[bi] = rho_total;
      rho_total += (int64_t)4 << (2 * popc(b.support));
    }
  }
  cudaStream_t st = s->stream;
  const bool f32 = s->dtype == QS_C64;
  const uint64_t dim = 1ull << n;
  if (host_loss) QS_TRY(expect_raw(s->data, s->dtype, n, 1, o, s, host_loss));
  void* lam = work;
  QS_TRY(f32 ? apply_obs<float>(s->data, lam, n, o, st) : apply_obs<double>(s->data, lam, n, o, st));
  int dev = 0, sms = 0;
  QS_CUDA(cudaGetDevice(&dev));
  QS_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const size_t npart = gram_partials_doubles(sms);
  QS_TRY(ensure_ws(s, s->ws, sizeof(double) * (npart + (size_t)rho_total) + 256));
  double* partials = (double*)s->ws.ptr;
  double* rhos = partials + npart;
  // device pass: per block, rho (if it has parameters) then the uncompute; no host round trip
  std::vector<int> qubits;
  std::vector<cd> M;
  for (int bi = nb - 1; bi >= 0; --bi) {
    const Block& b = blocks[bi];
    qubits.clear();
    for (int q = 0; q < 64; ++q)
      if ((b.support >> q) & 1ull) qubits.push_back(q);
    const int w = (int)qubits.size();
    if (rho_off[bi] >= 0) {
      if (f32 && (w == 4 || w == 5) && tensor_cores_enabled()) {
        int grid = 0;
        QS_TRY(gram_tc(w, (const float2*)s->data, (const float2*)lam, n, qubits.data(), partials, &grid, st));
        const int E = 4 << (2 * w);
        k_gram_fold<<<E, 256, 0, st>>>(partials, grid, E, rhos + rho_off[bi]);
        QS_LAUNCHED();
        rho_tc[bi] = 1;
      } else {
        QS_TRY(f32 ? gram<float>(w, s->data, lam, n, qubits, partials, rhos + rho_off[bi], st)
                   : gram<double>(w, s->data, lam, n, qubits, partials, rhos + rho_off[bi], st));
      }
    }
    Plan p;
    if (b.gates.size() == 1) {
      const qs_gate_desc& g = c->gates[b.gates[0]];
      QS_TRY(gate_matrix(c, g, params, M));
      dagger(M, g.nlocs);
      QS_TRY(plan_gate(M.data(), g.nlocs, g.locs, g.ctrl_mask, g.ctrl_vals, &p));
    } else {
      QS_TRY(block_matrix(c, b, params, qubits, M));
      dagger(M, w);
      QS_TRY(plan_gate(M.data(), w, qubits.data(), 0, 0, &p));
    }
    QS_TRY(launch_plan_on(s->data, s->dtype, n, 1, (int64_t)dim, p, s));
    QS_TRY(launch_plan_on(lam, s->dtype, n, 1, (int64_t)dim, p, s));
  }
  std::vector<double> G2((size_t)std::max<int64_t>(1, rho_total));
  if (rho_total > 0)
    QS_CUDA(cudaMemcpyAsync(G2.data(), rhos, sizeof(double) * rho_total, cudaMemcpyDeviceToHost, st));
  QS_CUDA(cudaStreamSynchronize(st));
  QS_TRY(tc_status_take());
  // host: every block's gradients from its rho (FP64)
  std::vector<double> grad(std::max(1, c->nparams), 0.0);
  std::vector<cd> U, H, Hemb, rho;
  for (int bi = 0; bi < nb; ++bi) {
    if (rho_off[bi] < 0) continue;
    const Block& b = blocks[bi];
    qubits.clear();
    for (int q = 0; q < 64; ++q)
      if ((b.support >> q) & 1ull) qubits.push_back(q);
    const int w = (int)qubits.size(), D = 1 << w, W2 = 2 * D;
    int pos[64];
    for (int j = 0; j < w; ++j) pos[qubits[j]] = j;
    const double* g2 = G2.data() + rho_off[bi];
    // rho[p][q] = sum_x psi_x[p] conj(lambda_x[q]), from the real Gram matrix: G[re p][re q]
    // + G[im p][im q] + i (G[im p][re q] - G[re p][im q]); rows / columns are [re | im]
    // halves (CUDA-core kernel) or interleaved re, im (tensor-core kernel)
    auto re = [&](int p) { return rho_tc[bi] ? 2 * p : p; };
    auto im = [&](int p) { return rho_tc[bi] ? 2 * p + 1 : D + p; };
    rho.assign((size_t)D * D, cd(0));
    for (int p = 0; p < D; ++p)
      for (int q = 0; q < D; ++q)
        rho[(size_t)p * D + q] = cd(g2[(size_t)re(p) * W2 + re(q)] + g2[(size_t)im(p) * W2 + im(q)],
                                    g2[(size_t)im(p) * W2 + re(q)] - g2[(size_t)re(p) * W2 + im(q)]);
    // from the last gate back: rho <- E^dag rho E with E the block's later gates, so that
    // Tr(E H E^dag rho) = Tr(H rho)
    for (int gj = (int)b.gates.size() - 1; gj >= 0; --gj) {
      const qs_gate_desc& g = c->gates[b.gates[gj]];
      int tpos[QS_MAXK];
      for (int j = 0; j < g.nlocs; ++j) tpos[j] = pos[g.locs[j]];
      uint32_t cmask = 0, cval = 0;
      for (int q = 0; q < 64; ++q)
        if ((g.ctrl_mask >> q) & 1ull) {
          cmask |= 1u << pos[q];
          if ((g.ctrl_vals >> q) & 1ull) cval |= 1u << pos[q];
        }
      if (g.param >= 0 && g.kind != QS_GATE_MATRIX) {
        double cfac = 0;
        QS_TRY(gate_generator(g, H, &cfac));
        embed_generator(H, g.nlocs, tpos, cmask, cval, w, Hemb);
        cd tr = 0;
        for (int i = 0; i < D; ++i)
          for (int j = 0; j < D; ++j) {
            const cd h = Hemb[(size_t)i * D + j];
            if (h != cd(0)) tr += h * rho[(size_t)j * D + i];
          }
        grad[g.param] += 2.0 * cfac * tr.imag();
      }
      if (gj > 0) {
        QS_TRY(gate_matrix(c, g, params, U));
        conj_by_gate(rho, w, U, g.nlocs, tpos, cmask, cval);
      }
    }
  }
  std::memcpy(host_grad, grad.data(), sizeof(double) * c->nparams);
  return QS_OK;
}

}  // namespace qs

using namespace qs;

extern "C" {

int qs_backward_blocks_work_bytes(int nqubits, int dtype, size_t* out_bytes) {
  if (!out_bytes || nqubits < 1 || nqubits > QS_MAXQ) return fail(QS_EINVAL, "bad arguments");
  if (dtype != QS_C64 && dtype != QS_C128) return fail(QS_EINVAL, "bad dtype");
  *out_bytes = ((size_t)1 << nqubits) * (dtype == QS_C64 ? 8 : 16);
  return QS_OK;
}

int qs_backward_blocks(qs_state* s, const qs_circuit* c, const double* params, const qs_observable* o, int kmax,
                       void* dev_work, double* host_grad, double* host_loss) {
  if (!s || !c || !o) return fail(QS_EINVAL, "null handle");
  return backward_blocks(s, c, params, o, kmax, dev_work, host_grad, host_loss);
}

int qs_circuit_blocks(const qs_circuit* c, const double* params, int kmax, int* nblocks, int32_t* widths,
                      int32_t* locs, double* mats) {
  if (!c || !nblocks) return fail(QS_EINVAL, "null argument");
  if (kmax < 1 || kmax > QS_MAXK) return fail(QS_EINVAL, "block width %d not in 1..%d", kmax, QS_MAXK);
  if (c->nparams > 0 && mats && !params) return fail(QS_EINVAL, "params is NULL");
  const std::vector<Block>& blocks = cached_blocks(c, kmax);
  *nblocks = (int)blocks.size();
  std::vector<int> qubits;
  std::vector<cd> M;
  const size_t stride = (size_t)1 << (2 * QS_MAXK);
  for (size_t i = 0; i < blocks.size(); ++i) {
    uint64_t sup = blocks[i].support;
    if (widths) widths[i] = popc(sup);
    if (locs) {
      int j = 0;
      for (int q = 0; q < 64; ++q)
        if ((sup >> q) & 1ull) {
          if (j < QS_MAXK) locs[i * QS_MAXK + j] = q;
          ++j;
        }
      for (; j < QS_MAXK; ++j) locs[i * QS_MAXK + j] = -1;
    }
    if (mats) {
      if (popc(sup) > QS_MAXK) return fail(QS_EINVAL, "a gate is wider than QS_MAXK");
      QS_TRY(block_matrix(c, blocks[i], params, qubits, M));
      std::memset(mats + 2 * stride * i, 0, 2 * stride * sizeof(double));
      std::memcpy(mats + 2 * stride * i, M.data(), M.size() * sizeof(cd));
    }
  }
  return QS_OK;
}

int qs_autotune_circuit(qs_state* s, const qs_circuit* c, const double* params, int reps, int* best_flags,
                        int* ncand, int32_t* cand_flags, double* cand_ms) {
  if (!s || !c || !best_flags) return fail(QS_EINVAL, "null argument");
  if (reps < 1) reps = 1;
  std::vector<int> cands = {QS_APPLY_UNFUSED, 0};
  for (int k = 2; k <= QS_MAXK; ++k) cands.push_back(QS_APPLY_BLOCKS | QS_APPLY_BLOCK_QUBITS(k));
  if (s->dtype == QS_C64 && s->uniform && s->nq[0] == c->nqubits)
    for (int m = 10; m <= 13; ++m)
      if (m <= s->nq[0]) cands.push_back(QS_APPLY_TILES | QS_APPLY_TILE_QUBITS(m));
  int best = -1;
  double best_ms = 0;
  for (size_t i = 0; i < cands.size(); ++i) {
    double ms = -1;
    int rc = qs_apply_circuit(s, c, params, cands[i]);  // warm-up (and plan caches)
    if (rc == QS_OK) rc = qs_state_sync(s);
    if (rc == QS_OK) {
      const auto t0 = std::chrono::steady_clock::now();
      for (int r = 0; r < reps && rc == QS_OK; ++r) rc = qs_apply_circuit(s, c, params, cands[i]);
      if (rc == QS_OK) rc = qs_state_sync(s);
      const auto t1 = std::chrono::steady_clock::now();
      if (rc == QS_OK) ms = std::chrono::duration<double, std::milli>(t1 - t0).count() / reps;
    }
    if (rc != QS_OK && rc != QS_EUNSUPPORTED) return rc;
    if (cand_flags && ncand && (int)i < *ncand) cand_flags[i] = cands[i];
    if (cand_ms && ncand && (int)i < *ncand) cand_ms[i] = ms;
    if (ms >= 0 && (best < 0 || ms < best_ms)) {
      best = cands[i];
      best_ms = ms;
    }
  }
  if (ncand) *ncand = (int)cands.size();
  if (best < 0) return fail(QS_EUNSUPPORTED, "no candidate applied the circuit");
  *best_flags = best;
  return QS_OK;
}

}  // extern "C"
