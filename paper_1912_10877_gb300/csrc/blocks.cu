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
// The planner walks the gates in order and keeps several open blocks with
// pairwise disjoint supports (so they commute).  A gate joins the open blocks
// it touches when the union of their supports and its own qubits (targets and
// controls) has at most k qubits; otherwise those blocks are emitted and the
// gate opens a new one.  The structure depends only on the gate list; the
// matrices are formed for each parameter vector.
#include <chrono>
#include <cstring>

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
    std::vector<Block> rest;
    for (Block& b : open) {
      if (b.support & q) out.push_back(std::move(b));
      else rest.push_back(std::move(b));
    }
    Block nb;
    nb.support = q;
    nb.gates.push_back(gi);
    if (popc(q) > kmax) out.push_back(std::move(nb));  // wider than k: stays a gate of its own
    else rest.push_back(std::move(nb));
    open.swap(rest);
  }
  for (Block& b : open) out.push_back(std::move(b));
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

int apply_blocks(qs_state* s, const qs_circuit* c, const double* params, int kmax) {
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
    QS_TRY(launch_plan(s, p));
  }
  return QS_OK;
}

}  // namespace qs

using namespace qs;

extern "C" {

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
