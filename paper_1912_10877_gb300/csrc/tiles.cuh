// tiles.cuh -- fused-pass representation shared by the batched engine and the
// single-register fused path (sm_103a).
//
// A circuit is scheduled into PASSES.  A pass owns a set B of m register
// qubits (its tile bits): the state is cut into 2^(n-m) tiles of 2^m
// amplitudes that differ only in those bits, each tile is staged in shared
// memory, and every non-diagonal gate of the pass has its target in B.  A pass
// is cut into PHASES: a phase owns rb of the tile's bits (its register bits R,
// rb = 2..4, the fusion width: every gate on those qubits in the phase is
// applied to amplitudes held in registers); each of the 2^(m-rb) threads
// holds the 2^rb amplitudes of the tile that differ only in R in registers,
// applies the phase's gates there, and writes them back.  A thread knows the global index of its amplitudes, so a gate's
// controls outside R become a per-thread predicate, and a diagonal gate whose
// target is outside R becomes a per-thread factor.  The planner keeps gate
// order valid by moving a gate earlier only past gates that share no qubit
// with it.
#pragma once

#include "common.cuh"

namespace qs {

constexpr int kRB = 4;             // register bits per phase by default (16 amplitudes per thread); the most
constexpr int kMinRB = 2;          // the fewest
constexpr int kRowBits = 5;        // tile rows: 32 consecutive amplitudes (register qubits 0..4)
constexpr int kMaxTileBits = 13;
constexpr int kTileThreads = 1 << (kMaxTileBits - kRB);  // 512

// one gate inside a phase.  t, cmask and cval are phase-local (bits 0..rb-1 of
// the register index j); the gate's other controls are register qubits outside the
// phase, tested per thread on its global base index: (base & tmask) == tval.
struct TOp {
  uint8_t kind;   // TK_*
  uint8_t t;      // target: phase bit (0..3), or the register qubit for TK_DIAGOUT
  uint8_t cmask;  // phase-local control bits
  uint8_t cval;   // their required values
  uint8_t gen;    // backward ops: generator code (GEN_*), 0 = no parameter
  uint8_t shared; // backward ops: the parameter also appears in another op of the phase
  uint8_t var;    // forward ops: the specialised form (fwd_variant), one jump per op
  uint8_t pad;
  int32_t param;  // register-local parameter index (forward TK_DIAG16: table index), -1 = none
  float cfac2;    // 2 c for U = exp(-i theta c H)
  uint32_t tmask; // controls outside the phase (register qubit bits)
  uint32_t tval;
  uint32_t count; // TK_DIAGRUN: entries (param: the first, relative to the pass's drun0)
  float2 u[4];    // forward: U; backward: U^dagger (row-major 2x2)
};

// TK_RX: u0 = u3 = c (real), u1 = u2 = i s; TK_RY: u0 = u3 = c, u1 = -s, u2 = s;
// TK_DIAG16 (forward only): amplitude j of the phase *= table[param][j], the
// product of consecutive diagonal gates inside the phase (they commute);
// TK_DIAGOUT: diagonal gate whose target qubit is outside the phase: every
// amplitude of the thread takes the factor u0 or u3 by that qubit's value
// TK_DIAGRUN (forward, complex64 path): a run of diagonal gates without
// phase-local controls that all commute with the ops between them: each entry
// (DRun) multiplies, where its outside controls hold, the amplitudes whose phase
// bit t is 0 by one factor and those whose bit t is 1 by another (a scalar when
// its target is outside the phase); the products are formed per thread and
// applied to the amplitudes once
enum { TK_DENSE = 0, TK_SWAP = 1, TK_DIAG = 2, TK_RX = 3, TK_RY = 4, TK_DIAG16 = 5, TK_DIAGOUT = 6, TK_DIAGRUN = 7 };

struct DRun {
  uint32_t tmask, tval;  // its controls (register qubit bits), all outside the phase
  int32_t gate;          // gate spec index (the matrix is formed from the parameters on the device)
  uint32_t tq;           // target register qubit when outside the phase (scalar entry), else 0xffffffff
  float2 u0, u3;         // the gate's diagonal
};
enum { GEN_NONE = 0, GEN_X = 1, GEN_Y = 2, GEN_Z = 3, GEN_P1 = 4, GEN_I = 5 };

struct TPhase {
  uint8_t rpos[kRB];        // tile-local positions of the register bits (ascending; rb used)
  uint8_t tpos[12];         // tile-local positions of the thread bits (ascending)
  uint8_t tq[12];           // register qubits of the thread bits
  uint16_t sroff[1 << kRB]; // swz(register offset of amplitude j): slot = swz(base) ^ sroff[j]
  int32_t fop0, nfop;       // forward ops (fused), applied in order
  int32_t bop0, nbop;       // backward ops (unfused), applied in reverse order
  int32_t nshared;          // backward ops whose parameter another op of the phase shares
};

struct TPass {
  uint8_t tbits[16];        // register qubits of tile-local bits 0..m-1 (ascending)
  uint8_t gbits[32];        // register qubits of the tile-id bits (ascending)
  int32_t phase0, nphase;
  int32_t drun0, ndrun;     // the pass's TK_DIAGRUN entries
};

struct HostPhase {
  int rbits[kRB];           // register qubits of the phase (ascending; rb used)
  std::vector<int> gates;   // circuit gate indices in forward order
};

struct HostPass {
  std::vector<int> tbits;   // register qubits of the tile (ascending)
  std::vector<HostPhase> phases;
};

// Greedy commutation-aware scheduling: passes of m qubits (always containing
// register qubits 0..4, so tile rows are contiguous), phases of exactly rb of
// the pass's qubits.  Gates must be single-target; a non-diagonal gate's target
// lies in its phase, its controls and diagonal gates may be anywhere.  Returns
// QS_OK or QS_EUNSUPPORTED.
int plan_passes(const qs_circuit* c, int n, int m, int max_phase_ops, std::vector<HostPass>& out, int rb = kRB);

// diagonal gates (fit in any phase: they only multiply amplitudes)
bool gate_is_diagonal(const qs_circuit* c, const qs_gate_desc& g);

// tile-local positions of a phase's register bits and thread bits
void phase_positions(const HostPass& p, const HostPhase& ph, TPhase* out, int rb = kRB);

// swizzled shared-memory slot of tile-local amplitude l (spreads the 8-byte
// accesses of a half-warp over all banks for the phase patterns used here).
// It is linear over XOR, so swz(base | r) = swz(base) ^ swz(r) for disjoint bits.
__host__ __device__ __forceinline__ uint32_t swz(uint32_t l) { return l ^ ((l >> 5) & 15u); }

}  // namespace qs
