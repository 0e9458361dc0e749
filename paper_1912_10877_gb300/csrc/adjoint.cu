// adjoint.cu -- reversible-adjoint backward pass (sm_103a), Sec. "Reverse Mode".
//
// With lambda = dL/dpsi* (Wirtinger) = O psi_N, gates are walked from last to
// first.  With psi and lambda the states right after gate k, a gate
// U = exp(-i theta c H) contributes dL/dtheta = 2 c Im<lambda|H|psi> (H includes
// the control projector), and then both states are uncomputed,
// psi <- U^dag psi, lambda <- U^dag lambda (Eq. apply-back); the outer product
// of Eq. outer-product is never formed, only its contraction with H.
//
// Parameterised gates run one fused pass per gate: each thread loads the
// psi and lambda 2^k-tuples, adds Im sum_m conj(l_m) (G x)_m to its FP64
// partial, applies U^dag to both tuples and stores them.  Block partials land
// in scratch memory and one block folds them pairwise into grad[param] in
// stream order.  The uncompute runs in FP64 (complex128 work buffers) whatever
// the forward precision; checkpoints taken during the forward replace psi at
// segment boundaries so that uncompute drift cannot accumulate across segments.
#include <cmath>
#include <cstring>

#include "common.cuh"

namespace qs {

int expect_raw(const void* data, int dtype, int n, int nreg, const qs_observable* o, qs_state* ws_owner,
               double* host_out);
int apply_observable_c128(const double2* psi, double2* lam, int n, const qs_observable* o, cudaStream_t st);
int promote_to_c128(const void* in, int dtype, double2* out, uint64_t dim, cudaStream_t st);

constexpr int kAdjThreads = 256;
constexpr int kAdjMaxBlocks = 1216;  // 8 per SM on 152 SMs

template <int K>
struct AdjMat {
  double2 g[1 << (2 * K)];   // generator H on the targets
  double2 ud[1 << (2 * K)];  // U^dagger on the targets
  uint64_t off[1 << K];
};

// Where the gradient of a launch goes: grad[param] += scale * (sum of the CTAs'
// contributions).  Each CTA writes its partial; the CTA that arrives last at
// the counter folds them pairwise in index order (the order does not depend on
// which CTA is last), adds the result and resets the counter for the next
// launch on the stream: no separate fold launch per gate.
struct AdjOut {
  double* partials;   // [gridDim.x]
  unsigned* counter;  // 0 between launches
  double* grad;
  int param;
  double scale;
};

__device__ __forceinline__ void adj_finish(double acc, const AdjOut& out) {
  __shared__ double red[kAdjThreads / 32];
  __shared__ bool last;
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double v = 0.0;
    for (int w = 0; w < kAdjThreads / 32; ++w) v += red[w];
    out.partials[blockIdx.x] = v;
    __threadfence();
    last = atomicAdd(out.counter, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  __shared__ double buf[2048];
  static_assert(kAdjMaxBlocks <= 2048, "one fold buffer");
  for (int i = threadIdx.x; i < 2048; i += blockDim.x) buf[i] = i < (int)gridDim.x ? __ldcg(out.partials + i) : 0.0;
  __syncthreads();
  for (int w = 1024; w > 0; w >>= 1) {
    for (int i = threadIdx.x; i < w; i += blockDim.x) buf[i] += buf[i + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out.grad[out.param] += out.scale * buf[0];
    *out.counter = 0u;
  }
}

template <int K>
__global__ void __launch_bounds__(kAdjThreads)
k_adjoint_param(double2* __restrict__ psi, double2* __restrict__ lam, uint64_t nitems, IdxSpec s,
                const __grid_constant__ AdjMat<K> M, const AdjOut out) {
  constexpr int D = 1 << K;
  double acc = 0.0;
  for (uint64_t it = (uint64_t)blockIdx.x * kAdjThreads + threadIdx.x; it < nitems;
       it += (uint64_t)gridDim.x * kAdjThreads) {
    const uint64_t base = item_index(it, s);
    double2 x[D], l[D];
#pragma unroll
    for (int m = 0; m < D; ++m) {
      x[m] = psi[base + M.off[m]];
      l[m] = lam[base + M.off[m]];
    }
    // Im sum_m conj(l_m) (G x)_m
#pragma unroll
    for (int m = 0; m < D; ++m) {
      double2 gx = make_double2(0.0, 0.0);
#pragma unroll
      for (int j = 0; j < D; ++j) gx = cfma(M.g[m * D + j], x[j], gx);
      acc += l[m].x * gx.y - l[m].y * gx.x;
    }
#pragma unroll
    for (int m = 0; m < D; ++m) {
      double2 px = make_double2(0.0, 0.0), pl = make_double2(0.0, 0.0);
#pragma unroll
      for (int j = 0; j < D; ++j) {
        px = cfma(M.ud[m * D + j], x[j], px);
        pl = cfma(M.ud[m * D + j], l[j], pl);
      }
      psi[base + M.off[m]] = px;
      lam[base + M.off[m]] = pl;
    }
  }
  adj_finish(acc, out);
}

// Single-target parameterised gates in structured forms (FP64 is scarce on
// this part: the dense 2x2 path spends 64 FP64 multiply-adds per pair):
//   ADJ_DIAG: U^dag = diag(u0, u3), H = diag(g0, g3) real (Rz, shift, phase):
//             ~20 per pair;
//   ADJ_RX:   U^dag = [[c, i s], [i s, c]], H = X (Rx): ~24 per pair.
enum { ADJ_DIAG = 0, ADJ_RX = 1 };

struct AdjForm1 {
  double2 u0, u3;   // ADJ_DIAG: the diagonal of U^dag
  double g0, g3;    // ADJ_DIAG: the diagonal of H
  double c, s;      // ADJ_RX: U^dag = [[c, i s], [i s, c]]
  uint64_t off1;    // offset of the target bit
};

template <int FORM>
__global__ void __launch_bounds__(kAdjThreads)
k_adjoint_param1(double2* __restrict__ psi, double2* __restrict__ lam, uint64_t nitems, IdxSpec s,
                 const __grid_constant__ AdjForm1 F, const AdjOut out) {
  double acc = 0.0;
  for (uint64_t it = (uint64_t)blockIdx.x * kAdjThreads + threadIdx.x; it < nitems;
       it += (uint64_t)gridDim.x * kAdjThreads) {
    const uint64_t b0 = item_index(it, s), b1 = b0 + F.off1;
    double2 x0 = psi[b0], x1 = psi[b1], l0 = lam[b0], l1 = lam[b1];
    if (FORM == ADJ_DIAG) {
      // Im conj(l) H x with H diagonal and real
      acc = fma(F.g0, fma(l0.x, x0.y, -l0.y * x0.x), acc);
      acc = fma(F.g3, fma(l1.x, x1.y, -l1.y * x1.x), acc);
      x0 = cmul(F.u0, x0);
      x1 = cmul(F.u3, x1);
      l0 = cmul(F.u0, l0);
      l1 = cmul(F.u3, l1);
    } else {
      // Im (conj(l0) x1 + conj(l1) x0) for H = X
      acc += fma(l0.x, x1.y, -l0.y * x1.x) + fma(l1.x, x0.y, -l1.y * x0.x);
      const double c = F.c, sn = F.s;
      const double2 nx0 = make_double2(fma(c, x0.x, -sn * x1.y), fma(c, x0.y, sn * x1.x));
      const double2 nx1 = make_double2(fma(c, x1.x, -sn * x0.y), fma(c, x1.y, sn * x0.x));
      const double2 nl0 = make_double2(fma(c, l0.x, -sn * l1.y), fma(c, l0.y, sn * l1.x));
      const double2 nl1 = make_double2(fma(c, l1.x, -sn * l0.y), fma(c, l1.y, sn * l0.x));
      x0 = nx0; x1 = nx1; l0 = nl0; l1 = nl1;
    }
    psi[b0] = x0;
    psi[b1] = x1;
    lam[b0] = l0;
    lam[b1] = l1;
  }
  adj_finish(acc, out);
}

// the structured form of a single-target gate, or -1
static int adj_form1(const std::vector<cd>& G, const std::vector<cd>& Ud, AdjForm1* F) {
  const cd z(0, 0);
  if (G[1] == z && G[2] == z && G[0].imag() == 0 && G[3].imag() == 0 && Ud[1] == z && Ud[2] == z) {
    F->u0 = make_double2(Ud[0].real(), Ud[0].imag());
    F->u3 = make_double2(Ud[3].real(), Ud[3].imag());
    F->g0 = G[0].real();
    F->g3 = G[3].real();
    return ADJ_DIAG;
  }
  if (G[0] == z && G[3] == z && G[1] == cd(1, 0) && G[2] == cd(1, 0) && Ud[0] == Ud[3] && Ud[0].imag() == 0 &&
      Ud[1] == Ud[2] && Ud[1].real() == 0) {
    F->c = Ud[0].real();
    F->s = Ud[1].imag();
    return ADJ_RX;
  }
  return -1;
}

template <int K>
static int launch_adjoint_param(double2* psi, double2* lam, int n, const qs_gate_desc& g,
                                const std::vector<cd>& G, const std::vector<cd>& Ud, double* partials,
                                unsigned* counter, double* dgrad, double cfac, cudaStream_t st) {
  const AdjOut out{partials, counter, dgrad, g.param, 2.0 * cfac};
  if constexpr (K == 1) {
    AdjForm1 F;
    memset(&F, 0, sizeof(F));
    const int form = adj_form1(G, Ud, &F);
    if (form >= 0) {
      F.off1 = 1ull << g.locs[0];
      IdxSpec s;
      QS_TRY(make_idx(n, F.off1 | g.ctrl_mask, g.ctrl_vals & g.ctrl_mask, &s));
      const uint64_t items = 1ull << s.item_log2;
      const int nblk = (int)std::min<uint64_t>(kAdjMaxBlocks, std::max<uint64_t>(1, (items + kAdjThreads * 4 - 1) / (kAdjThreads * 4)));
      if (form == ADJ_DIAG)
        k_adjoint_param1<ADJ_DIAG><<<nblk, kAdjThreads, 0, st>>>(psi, lam, items, s, F, out);
      else
        k_adjoint_param1<ADJ_RX><<<nblk, kAdjThreads, 0, st>>>(psi, lam, items, s, F, out);
      QS_LAUNCHED();
      return QS_OK;
    }
  }
  AdjMat<K> M;
  memset(&M, 0, sizeof(M));
  constexpr int D = 1 << K;
  uint64_t locmask = 0;
  for (int j = 0; j < K; ++j) locmask |= 1ull << g.locs[j];
  for (int m = 0; m < D; ++m) {
    uint64_t o = 0;
    for (int j = 0; j < K; ++j)
      if ((m >> j) & 1) o |= 1ull << g.locs[j];
    M.off[m] = o;
  }
  for (int i = 0; i < D * D; ++i) {
    M.g[i] = make_double2(G[i].real(), G[i].imag());
    M.ud[i] = make_double2(Ud[i].real(), Ud[i].imag());
  }
  IdxSpec s;
  QS_TRY(make_idx(n, locmask | g.ctrl_mask, g.ctrl_vals & g.ctrl_mask, &s));
  const uint64_t items = 1ull << s.item_log2;
  const int nblk = (int)std::min<uint64_t>(kAdjMaxBlocks, std::max<uint64_t>(1, (items + kAdjThreads * 4 - 1) / (kAdjThreads * 4)));
  k_adjoint_param<K><<<nblk, kAdjThreads, 0, st>>>(psi, lam, items, s, M, out);
  QS_LAUNCHED();
  return QS_OK;
}

// generator H (on the targets) and factor c with U = exp(-i theta c H)
int gate_generator(const qs_gate_desc& g, std::vector<cd>& G, double* cfac) {
  const int D = 1 << g.nlocs;
  G.assign(D * D, cd(0, 0));
  switch (g.kind) {
    case QS_GATE_RX: G[1] = 1; G[2] = 1; *cfac = 0.5; return QS_OK;
    case QS_GATE_RY: G[1] = cd(0, -1); G[2] = cd(0, 1); *cfac = 0.5; return QS_OK;
    case QS_GATE_RZ: G[0] = 1; G[3] = -1; *cfac = 0.5; return QS_OK;
    case QS_GATE_SHIFT: G[3] = 1; *cfac = -1.0; return QS_OK;
    case QS_GATE_PHASE: G[0] = 1; G[3] = 1; *cfac = -1.0; return QS_OK;
    case QS_GATE_ROT:
      pauli_string(g.nlocs, g.paulis, G);
      *cfac = 0.5;
      return QS_OK;
  }
  return fail(QS_EUNSUPPORTED, "gate kind %d has no parameter gradient", g.kind);
}

int backward(qs_state* s, const qs_circuit* c, const double* params, const qs_observable* o, int ckpt_every,
             const void* ckpts, void* work, double* host_grad, double* host_loss) {
  if (s->nreg != 1) return fail(QS_EUNSUPPORTED, "qs_backward takes a single register");
  const int n = s->nq[0];
  if (n != c->nqubits) return fail(QS_EINVAL, "circuit has %d qubits, state %d", c->nqubits, n);
  if (ckpt_every < 0 || (ckpt_every > 0 && !ckpts)) return fail(QS_EINVAL, "bad checkpoint arguments");
  if (!work) return fail(QS_EINVAL, "work buffer is NULL");
  cudaStream_t st = s->stream;
  const uint64_t dim = 1ull << n;
  double2* psi = (double2*)work;
  double2* lam = psi + dim;
  const int np = std::max(1, c->nparams);
  if (host_loss) QS_TRY(expect_raw(s->data, s->dtype, n, 1, o, s, host_loss));
  // scratch: grad[np] | partials[kAdjMaxBlocks]
  QS_TRY(ensure_ws(s, s->ws, sizeof(double) * (np + kAdjMaxBlocks) + 256));
  double* dgrad = (double*)s->ws.ptr;
  double* partials = dgrad + np;
  unsigned* counter = reinterpret_cast<unsigned*>(partials + kAdjMaxBlocks);
  QS_CUDA(cudaMemsetAsync(dgrad, 0, sizeof(double) * np, st));
  QS_CUDA(cudaMemsetAsync(counter, 0, sizeof(unsigned), st));
  QS_TRY(promote_to_c128(s->data, s->dtype, psi, dim, st));
  QS_TRY(apply_observable_c128(psi, lam, n, o, st));
  const size_t ab = amp_bytes(s->dtype);
  std::vector<cd> U, G;
  for (int k = (int)c->gates.size() - 1; k >= 0; --k) {
    const qs_gate_desc& g = c->gates[k];
    if (ckpt_every > 0 && (k + 1) % ckpt_every == 0 && k + 1 < (int)c->gates.size()) {
      const int slot = (k + 1) / ckpt_every - 1;
      QS_TRY(promote_to_c128((const char*)ckpts + ab * dim * slot, s->dtype, psi, dim, st));
    }
    QS_TRY(gate_matrix(c, g, params, U));
    dagger(U, g.nlocs);
    if (g.param >= 0 && g.kind != QS_GATE_MATRIX) {
      double cfac = 0;
      QS_TRY(gate_generator(g, G, &cfac));
      int rc;
      switch (g.nlocs) {
        case 1: rc = launch_adjoint_param<1>(psi, lam, n, g, G, U, partials, counter, dgrad, cfac, st); break;
        case 2: rc = launch_adjoint_param<2>(psi, lam, n, g, G, U, partials, counter, dgrad, cfac, st); break;
        case 3: rc = launch_adjoint_param<3>(psi, lam, n, g, G, U, partials, counter, dgrad, cfac, st); break;
        default: rc = fail(QS_EUNSUPPORTED, "parameterised gate on %d targets", g.nlocs);
      }
      QS_TRY(rc);
    } else {
      // psi and lambda are adjacent in the work buffer: one launch over both as
      // a batch of two registers
      Plan p;
      QS_TRY(plan_gate(U.data(), g.nlocs, g.locs, g.ctrl_mask, g.ctrl_vals, &p));
      QS_TRY(launch_plan_on(psi, QS_C128, n, 2, dim, p, s));
    }
  }
  QS_CUDA(cudaMemcpyAsync(host_grad, dgrad, sizeof(double) * c->nparams, cudaMemcpyDeviceToHost, st));
  QS_CUDA(cudaStreamSynchronize(st));
  return QS_OK;
}

}  // namespace qs

// ------------------------------------------------------------------ one gate of the adjoint walk
//
// qs_adjoint_step: the per-gate step of the walk above on two caller-held
// complex128 registers, for callers that walk a circuit themselves (the
// qubit-sharded register, whose gates may need data exchanges in between).

namespace qs {

// the matrix pool of a desc: MATRIX gates read 4^k entries at mat_offset
static int desc_matrix(const qs_gate_desc& g, const double* host_mats, const double* params, std::vector<cd>& U) {
  if (g.kind == QS_GATE_MATRIX) {
    if (!host_mats || g.mat_offset < 0) return fail(QS_EINVAL, "MATRIX gate without its matrix");
    const int D = 1 << g.nlocs;
    U.resize(D * D);
    for (int i = 0; i < D * D; ++i)
      U[i] = cd(host_mats[2 * (g.mat_offset + i)], host_mats[2 * (g.mat_offset + i) + 1]);
    return QS_OK;
  }
  qs_circuit tmp;
  tmp.nqubits = QS_MAXQ;
  return gate_matrix(&tmp, g, params, U);
}

static int check_desc(const qs_gate_desc& g, int n, const double* params) {
  int32_t locs[QS_MAXK];
  if (g.nlocs < 1 || g.nlocs > QS_MAXK) return fail(QS_EINVAL, "gate arity %d", g.nlocs);
  for (int j = 0; j < g.nlocs; ++j) locs[j] = g.locs[j];
  QS_TRY(validate_gate(n, g.nlocs, locs, g.ctrl_mask));
  if (g.param >= 0 && !params) return fail(QS_EINVAL, "the gate needs the parameter vector");
  return QS_OK;
}

}  // namespace qs

using namespace qs;

extern "C" {

int qs_gate_desc_matrices(const qs_gate_desc* g, const double* host_mats, const double* host_params, int dagger_u,
                          double* host_U, double* host_G, double* host_cfac) {
  if (!g) return fail(QS_EINVAL, "null gate");
  QS_TRY(check_desc(*g, QS_MAXQ, host_params));
  const int D = 1 << g->nlocs;
  if (host_U) {
    std::vector<cd> U;
    QS_TRY(desc_matrix(*g, host_mats, host_params, U));
    if (dagger_u) dagger(U, g->nlocs);
    for (int i = 0; i < D * D; ++i) { host_U[2 * i] = U[i].real(); host_U[2 * i + 1] = U[i].imag(); }
  }
  if (host_G || host_cfac) {
    if (g->param < 0) return fail(QS_EINVAL, "the gate has no parameter");
    std::vector<cd> G;
    double cf = 0.0;
    QS_TRY(gate_generator(*g, G, &cf));
    if (host_G)
      for (int i = 0; i < D * D; ++i) { host_G[2 * i] = G[i].real(); host_G[2 * i + 1] = G[i].imag(); }
    if (host_cfac) *host_cfac = cf;
  }
  return QS_OK;
}

int qs_adjoint_step(qs_state* psi, qs_state* lam, const qs_gate_desc* g, const double* host_mats,
                    const double* host_params, double* dev_grad) {
  if (!psi || !lam || !g) return fail(QS_EINVAL, "null argument");
  if (psi->dtype != QS_C128 || lam->dtype != QS_C128) return fail(QS_EINVAL, "qs_adjoint_step takes complex128 states");
  if (psi->nreg != 1 || lam->nreg != 1 || psi->nq[0] != lam->nq[0])
    return fail(QS_EINVAL, "psi and lambda must be single registers of one size");
  if (psi->data == lam->data) return fail(QS_EINVAL, "psi and lambda must be distinct");
  const int n = psi->nq[0];
  QS_TRY(check_desc(*g, n, host_params));
  const bool param = g->param >= 0 && g->kind != QS_GATE_MATRIX;
  if (param && !dev_grad) return fail(QS_EINVAL, "dev_grad is NULL");
  cudaStream_t st = psi->stream;
  std::vector<cd> U;
  QS_TRY(desc_matrix(*g, host_mats, host_params, U));
  dagger(U, g->nlocs);
  double2* x = (double2*)psi->data;
  double2* l = (double2*)lam->data;
  if (!param) {
    Plan p;
    QS_TRY(plan_gate(U.data(), g->nlocs, g->locs, g->ctrl_mask, g->ctrl_vals, &p));
    QS_TRY(launch_plan_on(x, QS_C128, n, 1, 1ll << n, p, psi));
    QS_TRY(launch_plan_on(l, QS_C128, n, 1, 1ll << n, p, psi));
    return QS_OK;
  }
  std::vector<cd> G;
  double cfac = 0.0;
  QS_TRY(gate_generator(*g, G, &cfac));
  QS_TRY(ensure_ws(psi, psi->ws, sizeof(double) * kAdjMaxBlocks + 256));
  double* partials = (double*)psi->ws.ptr;
  unsigned* counter = reinterpret_cast<unsigned*>(partials + kAdjMaxBlocks);
  QS_CUDA(cudaMemsetAsync(counter, 0, sizeof(unsigned), st));
  switch (g->nlocs) {
    case 1: return launch_adjoint_param<1>(x, l, n, *g, G, U, partials, counter, dev_grad, cfac, st);
    case 2: return launch_adjoint_param<2>(x, l, n, *g, G, U, partials, counter, dev_grad, cfac, st);
    case 3: return launch_adjoint_param<3>(x, l, n, *g, G, U, partials, counter, dev_grad, cfac, st);
  }
  return fail(QS_EUNSUPPORTED, "parameterised gate on %d targets", g->nlocs);
}

int qs_sample_shards(int nshards, const double* host_weights, int nshots, const double* host_u,
                     int32_t* host_shard, double* host_u_in_shard) {
  if (nshards < 1 || nshots < 0 || !host_weights || (nshots > 0 && (!host_u || !host_shard || !host_u_in_shard)))
    return fail(QS_EINVAL, "bad arguments");
  // the walk of qs_measure's contract over the shard weights: T = left fold of
  // the weights, t = u T, first shard whose running sum exceeds t (else the last
  // positive weight, else the last shard); its exclusive prefix a gives the
  // uniform of the shard's own sampler u' = (t - a) / P_s, kept below 1
  double total = host_weights[0];
  for (int s = 1; s < nshards; ++s) total = total + host_weights[s];
  for (int i = 0; i < nshots; ++i) {
    if (!(host_u[i] >= 0.0 && host_u[i] < 1.0)) return fail(QS_EINVAL, "uniform %d not in [0, 1)", i);
    const double t = host_u[i] * total;
    double a = 0.0, a_last = 0.0;
    int pick = -1, last = -1;
    for (int s = 0; s < nshards; ++s) {
      const double nxt = a + host_weights[s];
      if (nxt > t) { pick = s; break; }
      if (host_weights[s] > 0.0) { last = s; a_last = a; }
      a = nxt;
    }
    if (pick < 0) {
      if (last >= 0) { pick = last; a = a_last; }
      else { pick = nshards - 1; }
    }
    const double w = host_weights[pick];
    double v = w > 0.0 ? (t - a) / w : 0.0;
    if (!(v >= 0.0)) v = 0.0;
    if (v >= 1.0) v = std::nextafter(1.0, 0.0);
    host_shard[i] = pick;
    host_u_in_shard[i] = v;
  }
  return QS_OK;
}

}  // extern "C"

