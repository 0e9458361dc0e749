// api.cu -- the C ABI of include/qsim.h: argument validation, object lifetime,
// and the host-side circuit walk (gate matrices, same-qubit fusion, launches).
// The register and instruction model is that of Sec. "Quantum Registers" and
// Sec. "Instructions on Quantum Registers"; apply! of a chain follows Sec.
// "Representing Quantum Circuits" (gates in list order; consecutive
// single-qubit gates on one qubit are multiplied into one 2x2 first).
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstring>

#include "common.cuh"

namespace qs {

static thread_local std::string g_err;

void set_error(const char* fmt, ...) {
  char buf[1024];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_err = buf;
}

int fail(int code, const char* fmt, ...) {
  char buf[1024];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}

int ensure_ws(qs_state* s, Workspace& w, size_t bytes) {
  if (w.bytes >= bytes) return QS_OK;
  if (w.ptr) {
    QS_CUDA(cudaStreamSynchronize(s->stream));
    QS_CUDA(cudaFree(w.ptr));
    w.ptr = nullptr;
    w.bytes = 0;
  }
  size_t want = std::max<size_t>(bytes, 1 << 16);
  if (cudaMalloc(&w.ptr, want) != cudaSuccess) {
    cudaGetLastError();
    w.ptr = nullptr;
    return fail(QS_ENOMEM, "cudaMalloc of %zu scratch bytes failed", want);
  }
  w.bytes = want;
  return QS_OK;
}

int expect_raw(const void* data, int dtype, int n, int nreg, const qs_observable* o, qs_state* ws_owner,
               double* host_out);
int measure_one(void* data, int dtype, int n, const double* host_u, int nshots, int64_t* host_out,
                int collapse, qs_state* owner, const uint64_t* seed, uint64_t k0);
int reset_basis(qs_state* s, const uint64_t* host_basis);
int backward(qs_state* s, const qs_circuit* c, const double* params, const qs_observable* o, int ckpt_every,
             const void* ckpts, void* work, double* host_grad, double* host_loss);

static int min_n(const qs_state* s) { return *std::min_element(s->nq.begin(), s->nq.end()); }

static int check_dtype(int dtype) {
  return (dtype == QS_C64 || dtype == QS_C128) ? QS_OK : fail(QS_EINVAL, "dtype must be QS_C64 or QS_C128");
}

static int make_state(int nreg, const int32_t* nq, int dtype, void* dev_buf, void* stream, qs_state** out) {
  if (!out) return fail(QS_EINVAL, "out is NULL");
  *out = nullptr;
  QS_TRY(check_dtype(dtype));
  if (nreg < 1) return fail(QS_EINVAL, "nreg must be >= 1");
  if (dev_buf && ((uintptr_t)dev_buf & 255)) return fail(QS_EINVAL, "dev_buf must be 256-byte aligned");
  qs_state* s = new qs_state();
  s->dtype = dtype;
  s->nreg = nreg;
  s->nq.resize(nreg);
  s->off.resize(nreg + 1);
  s->off[0] = 0;
  for (int r = 0; r < nreg; ++r) {
    if (nq[r] < 1 || nq[r] > QS_MAXQ) {
      delete s;
      return fail(QS_EINVAL, "register %d: nqubits %d not in 1..%d", r, nq[r], QS_MAXQ);
    }
    s->nq[r] = nq[r];
    s->off[r + 1] = s->off[r] + (1ll << nq[r]);
    if (nq[r] != nq[0]) s->uniform = false;
  }
  s->bytes = amp_bytes(dtype) * (size_t)s->off[nreg];
  s->stream = (cudaStream_t)stream;
  if (dev_buf) {
    s->data = dev_buf;
  } else {
    if (cudaMalloc(&s->data, s->bytes) != cudaSuccess) {
      cudaGetLastError();
      const size_t b = s->bytes;
      delete s;
      return fail(QS_ENOMEM, "cudaMalloc of %zu state bytes failed", b);
    }
    s->owns = true;
  }
  *out = s;
  return QS_OK;
}

// same-qubit single-qubit fusion: a pending 2x2 per qubit; gates that touch a
// qubit flush its pending matrix first (gates on other qubits commute with it)
struct Fuser {
  qs_state* s;
  std::vector<std::vector<cd>> pend;
  std::vector<bool> has;
  bool precise = false;
  explicit Fuser(qs_state* st, int n) : s(st), pend(n), has(n, false) {}
  int flush(int q) {
    if (!has[q]) return QS_OK;
    has[q] = false;
    Plan p;
    int loc = q;
    QS_TRY(plan_gate(pend[q].data(), 1, &loc, 0, 0, &p));
    p.precise = precise;
    return launch_plan(s, p);
  }
  int flush_mask(uint64_t m) {
    for (int q = 0; q < (int)has.size(); ++q)
      if ((m >> q) & 1ull) QS_TRY(flush(q));
    return QS_OK;
  }
  int flush_all() { return flush_mask(~0ull); }
  void push(int q, const std::vector<cd>& U) {
    if (!has[q]) {
      pend[q] = U;
      has[q] = true;
      return;
    }
    const std::vector<cd>& A = pend[q];  // new = U * A
    std::vector<cd> C = {U[0] * A[0] + U[1] * A[2], U[0] * A[1] + U[1] * A[3],
                         U[2] * A[0] + U[3] * A[2], U[2] * A[1] + U[3] * A[3]};
    pend[q] = C;
  }
};

static int apply_circuit_impl(qs_state* s, const qs_circuit* c, const double* params, int flags,
                              int ckpt_every, void* ckpts) {
  if (!s || !c) return fail(QS_EINVAL, "null handle");
  if (c->nparams > 0 && !params) return fail(QS_EINVAL, "params is NULL");
  if (min_n(s) < c->nqubits) return fail(QS_EINVAL, "circuit has %d qubits, register only %d", c->nqubits, min_n(s));
  const int ng = (int)c->gates.size();
  const bool per_register = (flags & QS_APPLY_PER_REGISTER) != 0;
  const bool unfused = (flags & QS_APPLY_UNFUSED) != 0;
  const bool per_gate = unfused || ckpt_every > 0;  // no tile engine or blocks
  // compensated gates on complex64: asked for, or the checkpointed forward
  // that feeds the FP64 reversible backward
  const bool precise = ((flags & QS_APPLY_PRECISE) != 0 || ckpt_every > 0) && s->dtype == QS_C64;
  std::vector<cd> U;
  if (per_register && s->nreg > 1) {
    if (!s->uniform) return fail(QS_EUNSUPPORTED, "per-register parameters on an uneven batch");
    // one register at a time (the batched persistent kernel is the fast path for this)
    const size_t ab = amp_bytes(s->dtype);
    for (int r = 0; r < s->nreg; ++r) {
      qs_state view = *s;
      view.nreg = 1;
      view.nq = {s->nq[r]};
      view.off = {0, 1ll << s->nq[r]};
      view.data = (char*)s->data + ab * s->off[r];
      view.owns = false;
      view.ws = Workspace();
      int rc = apply_circuit_impl(&view, c, params + (size_t)r * c->nparams, flags & ~QS_APPLY_PER_REGISTER, 0,
                                  nullptr);
      if (rc) return rc;
    }
    return QS_OK;
  }
  // tile engine: whole circuit in fused passes when it has enough tiles to fill the GPU
  const int tile = (flags >> 8) & 0xff;
  const bool force_tiles = (flags & QS_APPLY_TILES) != 0;
  if (force_tiles && (flags & QS_APPLY_BLOCKS)) return fail(QS_EINVAL, "QS_APPLY_TILES and QS_APPLY_BLOCKS together");
  if ((flags & QS_APPLY_PRECISE) && force_tiles)
    return fail(QS_EINVAL, "QS_APPLY_PRECISE runs the per-gate or block path (not with QS_APPLY_TILES)");
  if (!per_gate && !precise && !(flags & QS_APPLY_BLOCKS) && s->dtype == QS_C64 && s->uniform &&
      s->nq[0] == c->nqubits) {
    const int m = std::min(s->nq[0], tile > 0 ? tile : 13);
    const uint64_t tiles = (uint64_t)s->nreg << (s->nq[0] - m);
    if (force_tiles || tiles >= 256) {
      const int rc = fused_forward(s, c, params, tile);
      if (rc == QS_OK || rc != QS_EUNSUPPORTED || force_tiles) return rc;
    }
  } else if (force_tiles) {
    return fail(QS_EUNSUPPORTED, "the tile engine runs uniform complex64 registers of the circuit's size");
  }
  if ((flags & QS_APPLY_BLOCKS) && !per_gate) {
    const int kb = (flags >> 16) & 0xf;
    return apply_blocks(s, c, params, kb > 0 ? kb : QS_MAXK, precise);
  }
  Fuser fz(s, c->nqubits);
  fz.precise = precise;
  const size_t ab = amp_bytes(s->dtype);
  for (int k = 0; k < ng; ++k) {
    const qs_gate_desc& g = c->gates[k];
    QS_TRY(gate_matrix(c, g, params, U));
    uint64_t locmask = 0;
    for (int j = 0; j < g.nlocs; ++j) locmask |= 1ull << g.locs[j];
    if (g.nlocs == 1 && g.ctrl_mask == 0 && !unfused) {
      fz.push(g.locs[0], U);
    } else {
      QS_TRY(fz.flush_mask(locmask | g.ctrl_mask));
      Plan p;
      QS_TRY(plan_gate(U.data(), g.nlocs, g.locs, g.ctrl_mask, g.ctrl_vals, &p));
      p.precise = precise;
      QS_TRY(launch_plan(s, p));
    }
    if (ckpt_every > 0 && (k + 1) % ckpt_every == 0 && k + 1 < ng) {
      QS_TRY(fz.flush_all());  // the checkpoint holds the state after gate k exactly
      const int slot = (k + 1) / ckpt_every - 1;
      QS_CUDA(cudaMemcpyAsync((char*)ckpts + ab * (size_t)s->off[1] * slot, s->data, ab * (size_t)s->off[1],
                              cudaMemcpyDeviceToDevice, s->stream));
    }
  }
  return fz.flush_all();
}

}  // namespace qs

using namespace qs;

extern "C" {

const char* qs_last_error(void) { return g_err.c_str(); }

int qs_state_bytes(int nreg, const int32_t* nq, int dtype, size_t* out) {
  if (!nq || !out || nreg < 1) return fail(QS_EINVAL, "bad arguments");
  QS_TRY(check_dtype(dtype));
  size_t total = 0;
  for (int r = 0; r < nreg; ++r) {
    if (nq[r] < 1 || nq[r] > QS_MAXQ) return fail(QS_EINVAL, "nqubits out of range");
    total += (size_t)1 << nq[r];
  }
  *out = total * amp_bytes(dtype);
  return QS_OK;
}

int qs_state_create(int nqubits, int dtype, int nbatch, void* dev_buf, void* stream, qs_state** out) {
  if (nbatch < 1) return fail(QS_EINVAL, "nbatch must be >= 1");
  std::vector<int32_t> nq(nbatch, nqubits);
  return make_state(nbatch, nq.data(), dtype, dev_buf, stream, out);
}

int qs_batch_create(int nreg, const int32_t* nq, int dtype, void* dev_buf, void* stream, qs_state** out) {
  if (!nq) return fail(QS_EINVAL, "nqubits is NULL");
  return make_state(nreg, nq, dtype, dev_buf, stream, out);
}

int qs_state_destroy(qs_state* s) {
  if (!s) return QS_OK;
  cudaStreamSynchronize(s->stream);
  if (s->owns && s->data) cudaFree(s->data);
  if (s->ws.ptr) cudaFree(s->ws.ptr);
  delete s;
  return QS_OK;
}

int qs_state_set_stream(qs_state* s, void* stream) {
  if (!s) return fail(QS_EINVAL, "null state");
  QS_CUDA(cudaStreamSynchronize(s->stream));
  s->stream = (cudaStream_t)stream;
  return QS_OK;
}

int qs_state_data(const qs_state* s, void** dev_ptr, size_t* bytes, int64_t* offsets) {
  if (!s) return fail(QS_EINVAL, "null state");
  if (dev_ptr) *dev_ptr = s->data;
  if (bytes) *bytes = s->bytes;
  if (offsets)
    for (int r = 0; r <= s->nreg; ++r) offsets[r] = s->off[r];
  return QS_OK;
}

int qs_state_reset(qs_state* s, const uint64_t* basis) {
  if (!s) return fail(QS_EINVAL, "null state");
  return reset_basis(s, basis);
}

int qs_state_upload(qs_state* s, const void* host) {
  if (!s || !host) return fail(QS_EINVAL, "null argument");
  QS_CUDA(cudaMemcpyAsync(s->data, host, s->bytes, cudaMemcpyHostToDevice, s->stream));
  QS_CUDA(cudaStreamSynchronize(s->stream));
  return QS_OK;
}

int qs_state_download(const qs_state* s, void* host) {
  if (!s || !host) return fail(QS_EINVAL, "null argument");
  QS_CUDA(cudaMemcpyAsync(host, s->data, s->bytes, cudaMemcpyDeviceToHost, s->stream));
  QS_CUDA(cudaStreamSynchronize(s->stream));
  return QS_OK;
}

int qs_state_sync(qs_state* s) {
  if (!s) return fail(QS_EINVAL, "null state");
  QS_CUDA(cudaStreamSynchronize(s->stream));
  return tc_status_take();
}

int qs_set_option(int option, int value) {
  switch (option) {
    case QS_OPT_TENSOR_CORES: set_tensor_cores(value); return QS_OK;
  }
  return fail(QS_EINVAL, "unknown option %d", option);
}

int qs_get_option(int option, int* value) {
  if (!value) return fail(QS_EINVAL, "null argument");
  switch (option) {
    case QS_OPT_TENSOR_CORES: *value = tensor_cores_enabled(); return QS_OK;
  }
  return fail(QS_EINVAL, "unknown option %d", option);
}

static int ctrl_masks(int nctrl, const int32_t* cl, const int32_t* cv, uint64_t* mask, uint64_t* vals) {
  *mask = *vals = 0;
  if (nctrl < 0 || (nctrl > 0 && !cl)) return fail(QS_EINVAL, "bad control arguments");
  for (int i = 0; i < nctrl; ++i) {
    if (cl[i] < 0 || cl[i] >= 64) return fail(QS_EINVAL, "control loc %d out of range", cl[i]);
    if ((*mask >> cl[i]) & 1ull) return fail(QS_EINVAL, "duplicate control %d", cl[i]);
    *mask |= 1ull << cl[i];
    const int v = cv ? cv[i] : 1;
    if (v != 0 && v != 1) return fail(QS_EINVAL, "control value must be 0 or 1");
    if (v) *vals |= 1ull << cl[i];
  }
  return QS_OK;
}

static int apply_matrix(qs_state* s, const cd* U, int k, const int32_t* locs, uint64_t cm, uint64_t cv) {
  QS_TRY(validate_gate(min_n(s), k, locs, cm));
  Plan p;
  QS_TRY(plan_gate(U, k, locs, cm, cv, &p));
  return launch_plan(s, p);
}

int qs_apply_gate(qs_state* s, const double* mat, int k, const int32_t* locs, int nctrl, const int32_t* cl,
                  const int32_t* cv) {
  if (!s || !mat || !locs) return fail(QS_EINVAL, "null argument");
  if (k < 1 || k > QS_MAXK) return fail(QS_EINVAL, "k must be 1..%d", QS_MAXK);
  uint64_t cm, cvals;
  QS_TRY(ctrl_masks(nctrl, cl, cv, &cm, &cvals));
  const int D = 1 << k;
  std::vector<cd> U(D * D);
  for (int i = 0; i < D * D; ++i) U[i] = cd(mat[2 * i], mat[2 * i + 1]);
  return apply_matrix(s, U.data(), k, locs, cm, cvals);
}

int qs_apply_named(qs_state* s, int kind, int k, const int32_t* locs, const int32_t* paulis, int nctrl,
                   const int32_t* cl, const int32_t* cv, double theta) {
  if (!s || !locs) return fail(QS_EINVAL, "null argument");
  if (kind == QS_GATE_MATRIX) return fail(QS_EINVAL, "use qs_apply_gate for matrices");
  uint64_t cm, cvals;
  QS_TRY(ctrl_masks(nctrl, cl, cv, &cm, &cvals));
  std::vector<cd> U;
  QS_TRY(named_matrix(kind, k, paulis, theta, U));
  return apply_matrix(s, U.data(), k, locs, cm, cvals);
}

int qs_circuit_create(int nqubits, const qs_gate_desc* gates, int ngates, const double* mats, int64_t nmat,
                      int nparams, qs_circuit** out) {
  if (!out) return fail(QS_EINVAL, "out is NULL");
  *out = nullptr;
  if (nqubits < 1 || nqubits > QS_MAXQ) return fail(QS_EINVAL, "nqubits out of range");
  if (ngates < 0 || (ngates > 0 && !gates) || nparams < 0 || nmat < 0 || (nmat > 0 && !mats))
    return fail(QS_EINVAL, "bad arguments");
  qs_circuit* c = new qs_circuit();
  c->nqubits = nqubits;
  c->nparams = nparams;
  c->gates.assign(gates, gates + ngates);
  c->mats.resize(nmat);
  for (int64_t i = 0; i < nmat; ++i) c->mats[i] = cd(mats[2 * i], mats[2 * i + 1]);
  std::vector<cd> U;
  std::vector<double> zeros(std::max(1, nparams), 0.0);
  for (int k = 0; k < ngates; ++k) {
    const qs_gate_desc& g = c->gates[k];
    int rc = validate_gate(nqubits, g.nlocs, g.locs, g.ctrl_mask);
    if (!rc && (g.ctrl_vals & ~g.ctrl_mask)) rc = fail(QS_EINVAL, "gate %d: ctrl_vals outside ctrl_mask", k);
    if (!rc && g.param >= nparams) rc = fail(QS_EINVAL, "gate %d: param index %d >= nparams %d", k, g.param, nparams);
    if (!rc && g.param >= 0 && !(g.kind == QS_GATE_RX || g.kind == QS_GATE_RY || g.kind == QS_GATE_RZ ||
                                 g.kind == QS_GATE_SHIFT || g.kind == QS_GATE_PHASE || g.kind == QS_GATE_ROT))
      rc = fail(QS_EINVAL, "gate %d: kind %d takes no parameter", k, g.kind);
    if (!rc) rc = gate_matrix(c, g, zeros.data(), U);
    if (rc) {
      std::string msg = qs_last_error();
      delete c;
      return fail(rc, "gate %d: %s", k, msg.c_str());
    }
  }
  *out = c;
  return QS_OK;
}

int qs_circuit_destroy(qs_circuit* c) {
  if (c && c->fused) free_fused(c->fused);
  if (c) free_blocks(c);
  if (c) free_onelaunch(c);
  delete c;
  return QS_OK;
}

int qs_circuit_info(const qs_circuit* c, int* nq, int* ng, int* np) {
  if (!c) return fail(QS_EINVAL, "null circuit");
  if (nq) *nq = c->nqubits;
  if (ng) *ng = (int)c->gates.size();
  if (np) *np = c->nparams;
  return QS_OK;
}

int qs_circuit_schedule_info(const qs_circuit* c, int tile_qubits, int* npasses, int* nphases) {
  if (!c) return fail(QS_EINVAL, "null circuit");
  if (tile_qubits < 0 || tile_qubits > 13) return fail(QS_EINVAL, "tile_qubits must be 0 or 9..13");
  return schedule_info(c, tile_qubits, npasses, nphases);
}

int qs_circuit_tile_order(const qs_circuit* c, int tile_qubits, int* ngates, int32_t* host_order,
                          int32_t* host_pass) {
  if (!c || !ngates) return fail(QS_EINVAL, "null argument");
  if (tile_qubits < 0 || tile_qubits > 13) return fail(QS_EINVAL, "tile_qubits must be 0 or 9..13");
  std::vector<int> order, pass;
  QS_TRY(tile_order(c, tile_qubits, order, pass));
  *ngates = (int)order.size();
  for (size_t i = 0; i < order.size(); ++i) {
    if (host_order) host_order[i] = order[i];
    if (host_pass) host_pass[i] = pass[i];
  }
  return QS_OK;
}

int qs_apply_circuit(qs_state* s, const qs_circuit* c, const double* params, int flags) {
  return apply_circuit_impl(s, c, params, flags, 0, nullptr);
}

int qs_checkpoint_count(const qs_circuit* c, int every, int* count) {
  if (!c || !count || every < 0) return fail(QS_EINVAL, "bad arguments");
  const int ng = (int)c->gates.size();
  *count = every > 0 && ng > 0 ? (ng - 1) / every : 0;
  return QS_OK;
}

int qs_apply_circuit_ckpt(qs_state* s, const qs_circuit* c, const double* params, int every, void* ckpts) {
  if (!s || !c) return fail(QS_EINVAL, "null handle");
  if (s->nreg != 1) return fail(QS_EUNSUPPORTED, "checkpointed forward takes a single register");
  if (every < 0 || (every > 0 && !ckpts)) return fail(QS_EINVAL, "bad checkpoint arguments");
  return apply_circuit_impl(s, c, params, 0, every, ckpts);
}

int qs_observable_create(const qs_pauli_term* terms, int nterms, qs_observable** out) {
  if (!out || nterms < 0 || (nterms > 0 && !terms)) return fail(QS_EINVAL, "bad arguments");
  qs_observable* o = new qs_observable();
  o->terms.assign(terms, terms + nterms);
  *out = o;
  return QS_OK;
}

int qs_observable_destroy(qs_observable* o) {
  delete o;
  return QS_OK;
}

int qs_expect(qs_state* s, const qs_observable* o, double* out) {
  if (!s || !o || !out) return fail(QS_EINVAL, "null argument");
  if (s->uniform) return expect_raw(s->data, s->dtype, s->nq[0], s->nreg, o, s, out);
  const size_t ab = amp_bytes(s->dtype);
  for (int r = 0; r < s->nreg; ++r)
    QS_TRY(expect_raw((char*)s->data + ab * s->off[r], s->dtype, s->nq[r], 1, o, s, out + r));
  return QS_OK;
}

int qs_backward_work_bytes(int nqubits, size_t* out) {
  if (!out || nqubits < 1 || nqubits > QS_MAXQ) return fail(QS_EINVAL, "bad arguments");
  *out = (size_t)2 * 16 * ((size_t)1 << nqubits);
  return QS_OK;
}

int qs_backward(qs_state* s, const qs_circuit* c, const double* params, const qs_observable* o, int ckpt_every,
                const void* ckpts, void* work, double* grad, double* loss) {
  if (!s || !c || !o || !grad) return fail(QS_EINVAL, "null argument");
  if (c->nparams > 0 && !params) return fail(QS_EINVAL, "params is NULL");
  return backward(s, c, params, o, ckpt_every, ckpts, work, grad, loss);
}

int qs_backward_tiled_work_bytes(int nqubits, size_t* out) {
  if (!out || nqubits < 1 || nqubits > QS_MAXQ) return fail(QS_EINVAL, "bad arguments");
  *out = (size_t)2 * 8 * ((size_t)1 << nqubits);
  return QS_OK;
}

int qs_backward_tiled(qs_state* s, const qs_circuit* c, const double* params, const qs_observable* o,
                      int tile_qubits, void* work, double* grad, double* loss) {
  if (!s || !c || !o || (!grad && c->nparams > 0)) return fail(QS_EINVAL, "null argument");
  if (c->nparams > 0 && !params) return fail(QS_EINVAL, "params is NULL");
  if (tile_qubits < 0 || tile_qubits > 13) return fail(QS_EINVAL, "tile_qubits must be 0 or 9..13");
  return fused_backward(s, c, params, o, work, grad, loss, tile_qubits);
}

int qs_measure(qs_state* s, const double* u, int nshots, int64_t* out, int collapse) {
  if (!s || !u || !out) return fail(QS_EINVAL, "null argument");
  if (nshots < 1) return fail(QS_EINVAL, "nshots must be >= 1");
  if (collapse && nshots != 1) return fail(QS_EINVAL, "collapse needs nshots == 1");
  for (int i = 0; i < nshots * s->nreg; ++i)
    if (!(u[i] >= 0.0 && u[i] < 1.0)) return fail(QS_EINVAL, "uniform %d not in [0, 1)", i);
  const size_t ab = amp_bytes(s->dtype);
  for (int r = 0; r < s->nreg; ++r)
    QS_TRY(measure_one((char*)s->data + ab * s->off[r], s->dtype, s->nq[r], u + (size_t)r * nshots, nshots,
                       out + (size_t)r * nshots, collapse, s, nullptr, 0));
  return QS_OK;
}

int qs_measure_seeded(qs_state* s, uint64_t seed, int nshots, int64_t* out, int collapse) {
  if (!s || !out) return fail(QS_EINVAL, "null argument");
  if (nshots < 1) return fail(QS_EINVAL, "nshots must be >= 1");
  if (collapse && nshots != 1) return fail(QS_EINVAL, "collapse needs nshots == 1");
  const size_t ab = amp_bytes(s->dtype);
  for (int r = 0; r < s->nreg; ++r)
    QS_TRY(measure_one((char*)s->data + ab * s->off[r], s->dtype, s->nq[r], nullptr, nshots,
                       out + (size_t)r * nshots, collapse, s, &seed, (uint64_t)r * (uint64_t)nshots));
  return QS_OK;
}

}  // extern "C"
