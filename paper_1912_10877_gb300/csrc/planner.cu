// planner.cu -- host-side scheduling of a gate list into fused tile passes and
// register phases (see tiles.cuh).  Gates move earlier only past gates that
// share no qubit with them, so the schedule applies the same operator (a
// chain is the product of its parts in order, Sec. "Representing Quantum
// Circuits"; factors on disjoint qubits commute).  Only
// the target of a non-diagonal gate has to lie in the pass's tile and in the
// phase's register bits: controls are tested per thread on the global index,
// and a diagonal gate only multiplies amplitudes, so it fits anywhere.
#include <algorithm>
#include <cstring>

#include "tiles.cuh"

namespace qs {

static uint64_t qubits_of(const qs_gate_desc& g) {
  uint64_t q = g.ctrl_mask;
  for (int j = 0; j < g.nlocs; ++j) q |= 1ull << g.locs[j];
  return q;
}

bool gate_is_diagonal(const qs_circuit* c, const qs_gate_desc& g) {
  switch (g.kind) {
    case QS_GATE_I: case QS_GATE_Z: case QS_GATE_S: case QS_GATE_SDG: case QS_GATE_T: case QS_GATE_TDG:
    case QS_GATE_RZ: case QS_GATE_SHIFT: case QS_GATE_PHASE:
      return true;
    case QS_GATE_MATRIX:
      return g.nlocs == 1 && c->mats[g.mat_offset + 1] == cd(0, 0) && c->mats[g.mat_offset + 2] == cd(0, 0);
  }
  return false;
}

// greedy scan: take gates (in order) whose `fit` bits fit in `set` grown up to
// `cap` bits, skipping (and blocking all qubits of) gates that do not fit or
// depend on a skipped gate; at most `limit` gates are taken
static void scan(const std::vector<int>& rem, const std::vector<uint64_t>& dep, const std::vector<uint64_t>& fit,
                 uint64_t& set, int cap, size_t limit, std::vector<int>& taken, std::vector<int>& left) {
  uint64_t blocked = 0;
  for (int gi : rem) {
    if ((dep[gi] & blocked) || taken.size() >= limit) {
      blocked |= dep[gi];
      left.push_back(gi);
      continue;
    }
    const uint64_t u = set | fit[gi];
    if (__builtin_popcountll(u) <= cap) {
      set = u;
      taken.push_back(gi);
    } else {
      blocked |= dep[gi];
      left.push_back(gi);
    }
  }
}

static std::vector<int> bits_of(uint64_t m) {
  std::vector<int> v;
  for (int q = 0; q < 64; ++q)
    if ((m >> q) & 1ull) v.push_back(q);
  return v;
}

int plan_passes(const qs_circuit* c, int n, int m, int max_phase_ops, std::vector<HostPass>& out, int rb) {
  out.clear();
  if (m < kRowBits || m > n || m > kMaxTileBits)
    return fail(QS_EINVAL, "tile of %d qubits for a register of %d", m, n);
  if (rb < kMinRB || rb > kRB || rb > m) return fail(QS_EINVAL, "%d register bits per phase (tile of %d)", rb, m);
  const int G = (int)c->gates.size();
  std::vector<uint64_t> dep(G), fit(G);
  for (int i = 0; i < G; ++i) {
    const qs_gate_desc& g = c->gates[i];
    if (g.nlocs != 1)
      return fail(QS_EUNSUPPORTED, "gate %d: the fused tile engine takes single-target gates (kind %d, %d targets)",
                  i, g.kind, g.nlocs);
    dep[i] = qubits_of(g);
    fit[i] = gate_is_diagonal(c, g) ? 0ull : (1ull << g.locs[0]);
  }
  const uint64_t seed = (1ull << kRowBits) - 1ull;  // register qubits 0..4: contiguous tile rows
  std::vector<int> rem(G);
  for (int i = 0; i < G; ++i) rem[i] = i;
  while (!rem.empty()) {
    uint64_t B = seed;
    std::vector<int> taken, left;
    scan(rem, dep, fit, B, m, (size_t)-1, taken, left);
    if (taken.empty()) return fail(QS_EUNSUPPORTED, "no gate fits a %d-qubit tile", m);
    for (int b = 0; __builtin_popcountll(B) < m && b < n; ++b) B |= 1ull << b;  // pad with low qubits
    HostPass P;
    P.tbits = bits_of(B);
    std::vector<int> prem = taken;
    while (!prem.empty()) {
      uint64_t R = 0;
      std::vector<int> pt, pl;
      scan(prem, dep, fit, R, rb, (size_t)max_phase_ops, pt, pl);
      for (int b : P.tbits) {
        if (__builtin_popcountll(R) >= rb) break;
        R |= 1ull << b;
      }
      HostPhase ph;
      for (int k = 0; k < kRB; ++k) ph.rbits[k] = -1;
      std::vector<int> rbits = bits_of(R);
      for (int k = 0; k < rb; ++k) ph.rbits[k] = rbits[k];
      ph.gates = pt;
      P.phases.push_back(ph);
      prem.swap(pl);
    }
    out.push_back(std::move(P));
    rem.swap(left);
  }
  return QS_OK;
}

void phase_positions(const HostPass& p, const HostPhase& ph, TPhase* out, int rb) {
  memset(out, 0, sizeof(*out));
  const int m = (int)p.tbits.size();
  int nt = 0, nr = 0;
  for (int l = 0; l < m; ++l) {
    const int qb = p.tbits[l];
    bool inR = false;
    for (int k = 0; k < rb; ++k)
      if (ph.rbits[k] == qb) inR = true;
    if (inR) {
      out->rpos[nr++] = (uint8_t)l;
    } else {
      out->tq[nt] = (uint8_t)qb;
      out->tpos[nt++] = (uint8_t)l;
    }
  }
  for (int j = 0; j < (1 << rb); ++j) {
    uint32_t r = 0;
    for (int k = 0; k < rb; ++k)
      if ((j >> k) & 1) r |= 1u << out->rpos[k];
    out->sroff[j] = (uint16_t)swz(r);
  }
}

}  // namespace qs
