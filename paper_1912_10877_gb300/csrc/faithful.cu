// faithful.cu -- faithful (shot-based) expectation values and the
// parameter-shift gradient (Sec. "Forward Mode: Faithful Quantum Gradients",
// Eq. shiftrule).
//
// Shot-based <O> for a sum of Pauli strings: the terms are split into groups
// that share a measurement basis on every qubit (qubit-wise commuting; groups
// in order of first appearance in the term list, identity terms contribute
// their coefficient exactly).  For each group a copy of the state is rotated
// so that the group's X and Y qubits are measured in the computational basis
// (X: H; Y: S^dag then H, since H S^dag Y S H = Z), nshots basis indices are
// sampled per register with the library's deterministic sampler from the
// caller's uniforms, and each term's estimate is the mean over shots of
// (-1)^(number of 1s of the sample on the term's qubits).  The +-1 sums are
// exact integers; the estimate is c_t * sum / nshots in FP64, terms added in
// list order.
//
// The parameter-shift gradient runs the circuit at theta_k +- pi/2 for every
// parameter k (2 P registers in one batch), takes <O> at each (exact, or
// shot-based), and returns (<O>_+ - <O>_-) / 2.  It holds for parameters used
// by exactly one uncontrolled Pauli rotation (a reflexive generator).
//
// The MMD loss of a Born machine p_theta against a target distribution q,
// L = E_{x,x'~p} K(x,x') - 2 E_{x~p,y~q} K(x,y) + E_{y,y'~q} K(y,y'), with the
// Gaussian kernel K(x,y) = exp(-(x - y)^2 / (2 sigma^2)) on basis indices, has
// (from the paper's shift formula for order-two statistic functionals applied
// to both p-dependent terms) dL/dtheta_k = (p_+ - p_-)^T K (p - q), p_+- the
// output distributions at theta_k +- pi/2.  Exact mode uses |psi|^2; shot mode
// uses the empirical distributions of nshots samples per register (the
// plug-in estimate).  K acts as a convolution over the index difference,
// truncated where the kernel underflows to zero in FP64 (exact).
#include <cmath>
#include <cstring>

#include "common.cuh"

namespace qs {

namespace {

struct BasisGroup {
  uint64_t xq = 0, yq = 0, zq = 0;  // qubits measured in X, Y, Z
  std::vector<int> terms;
};

void group_terms(const qs_observable* o, std::vector<BasisGroup>& gs, double* constant) {
  gs.clear();
  *constant = 0;
  for (int t = 0; t < (int)o->terms.size(); ++t) {
    const qs_pauli_term& p = o->terms[t];
    const uint64_t X = p.x_mask & ~p.z_mask, Y = p.x_mask & p.z_mask, Z = p.z_mask & ~p.x_mask;
    if (!(X | Y | Z)) {
      *constant += p.coeff;
      continue;
    }
    bool placed = false;
    for (BasisGroup& g : gs) {
      if ((X & (g.yq | g.zq)) || (Y & (g.xq | g.zq)) || (Z & (g.xq | g.yq))) continue;
      g.xq |= X;
      g.yq |= Y;
      g.zq |= Z;
      g.terms.push_back(t);
      placed = true;
      break;
    }
    if (!placed) {
      BasisGroup g;
      g.xq = X;
      g.yq = Y;
      g.zq = Z;
      g.terms.push_back(t);
      gs.push_back(g);
    }
  }
}

constexpr int kEstTerms = 64;
struct EstTerms {
  int nt;
  uint64_t supp[kEstTerms];
  double coef[kEstTerms];
};

// out[r] += sum_t coef_t * (sum_s (-1)^popcount(x_rs & supp_t)) / nshots; one CTA per register
__global__ void __launch_bounds__(256) k_parity_estimate(const int64_t* __restrict__ samples, int nshots,
                                                         const __grid_constant__ EstTerms e, double* __restrict__ out) {
  __shared__ long long red[256];
  const int r = blockIdx.x;
  const int64_t* xs = samples + (size_t)r * nshots;
  double acc = 0.0;
  for (int t = 0; t < e.nt; ++t) {
    long long sum = 0;
    for (int s = threadIdx.x; s < nshots; s += 256) sum += (__popcll((unsigned long long)xs[s] & e.supp[t]) & 1) ? -1 : 1;
    red[threadIdx.x] = sum;
    __syncthreads();
    for (int h = 128; h > 0; h >>= 1) {
      if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
      __syncthreads();
    }
    if (threadIdx.x == 0) acc += e.coef[t] * ((double)red[0] / (double)nshots);
    __syncthreads();
  }
  if (threadIdx.x == 0) out[r] += acc;
}

int apply_1q_all(qs_state* view, int kind, int q) {
  std::vector<cd> U;
  QS_TRY(named_matrix(kind, 1, nullptr, 0.0, U));
  Plan p;
  QS_TRY(plan_gate(U.data(), 1, &q, 0, 0, &p));
  return launch_plan(view, p);
}

uint64_t obs_qubits(const qs_observable* o) {
  uint64_t m = 0;
  for (const qs_pauli_term& p : o->terms) m |= p.x_mask | p.z_mask;
  return m;
}

}  // namespace

int shot_expect(qs_state* s, const qs_observable* o, const double* host_u, int nshots, void* work, double* host_out) {
  std::vector<BasisGroup> gs;
  double constant = 0;
  group_terms(o, gs, &constant);
  int nmin = 64;
  for (int r = 0; r < s->nreg; ++r) nmin = std::min(nmin, s->nq[r]);
  const uint64_t oq = obs_qubits(o);
  if (nmin < 64 && (oq >> nmin)) return fail(QS_EINVAL, "observable acts on qubits beyond a register");
  if (!gs.empty() && (nshots < 1 || !host_u || !work)) return fail(QS_EINVAL, "shots, uniforms and work are needed");
  cudaStream_t st = s->stream;
  const int R = s->nreg;
  size_t sscr = 0;
  for (int r = 0; r < R; ++r) sscr = std::max(sscr, sample_scratch_doubles(s->nq[r]));
  const size_t nsr = (size_t)R * std::max(1, nshots);
  QS_TRY(ensure_ws(s, s->ws, sizeof(double) * (R + nsr + sscr) + sizeof(int64_t) * nsr + 256));
  double* dacc = (double*)s->ws.ptr;
  double* du = dacc + R;
  double* dscr = du + nsr;
  int64_t* dsamp = (int64_t*)(dscr + sscr);
  QS_CUDA(cudaMemsetAsync(dacc, 0, sizeof(double) * R, st));
  qs_state view = *s;
  view.data = work;
  view.owns = false;
  view.ws = Workspace();
  const size_t ab = amp_bytes(s->dtype);
  for (size_t g = 0; g < gs.size(); ++g) {
    const BasisGroup& G = gs[g];
    QS_CUDA(cudaMemcpyAsync(work, s->data, s->bytes, cudaMemcpyDeviceToDevice, st));
    for (int q = 0; q < 64; ++q) {
      if ((G.yq >> q) & 1ull) QS_TRY(apply_1q_all(&view, QS_GATE_SDG, q));
      if (((G.xq | G.yq) >> q) & 1ull) QS_TRY(apply_1q_all(&view, QS_GATE_H, q));
    }
    QS_CUDA(cudaMemcpyAsync(du, host_u + g * nsr, sizeof(double) * nsr, cudaMemcpyHostToDevice, st));
    for (int r = 0; r < R; ++r)
      QS_TRY(sample_dev((const char*)work + ab * s->off[r], s->dtype, s->nq[r], du + (size_t)r * nshots, nshots,
                        dsamp + (size_t)r * nshots, dscr, st));
    for (size_t t0 = 0; t0 < G.terms.size(); t0 += kEstTerms) {
      EstTerms e;
      std::memset(&e, 0, sizeof(e));
      e.nt = (int)std::min<size_t>(kEstTerms, G.terms.size() - t0);
      for (int i = 0; i < e.nt; ++i) {
        const qs_pauli_term& p = o->terms[G.terms[t0 + i]];
        e.supp[i] = p.x_mask | p.z_mask;
        e.coef[i] = p.coeff;
      }
      k_parity_estimate<<<R, 256, 0, st>>>(dsamp, nshots, e, dacc);
      QS_LAUNCHED();
    }
  }
  QS_CUDA(cudaMemcpyAsync(host_out, dacc, sizeof(double) * R, cudaMemcpyDeviceToHost, st));
  QS_CUDA(cudaStreamSynchronize(st));
  for (int r = 0; r < R; ++r) host_out[r] += constant;
  return QS_OK;
}

// ------------------------------------------------------------------ MMD loss

namespace {

// dist[r][x] = |psi_rx|^2 (FP64) for registers of 2^n amplitudes
template <typename T>
__global__ void k_probs(const T* __restrict__ psi, uint64_t total, double* __restrict__ dist) {
  const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= total) return;
  const double a = (double)psi[i].x, b = (double)psi[i].y;
  dist[i] = a * a + b * b;
}

// counts[r][x] = number of shots of register r that gave x (integer counts, zeroed before)
__global__ void k_hist(const int64_t* __restrict__ samples, int nshots, int nreg, uint64_t dim,
                       unsigned long long* __restrict__ counts) {
  const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (uint64_t)nreg * nshots) return;
  const uint64_t r = i / nshots;
  atomicAdd(counts + r * dim + (uint64_t)samples[i], 1ull);
}

// in place: dist = count / nshots (one correctly rounded division per entry)
__global__ void k_counts_to_dist(double* __restrict__ buf, uint64_t total, int nshots) {
  const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= total) return;
  const unsigned long long c = reinterpret_cast<const unsigned long long*>(buf)[i];
  buf[i] = (double)c / (double)nshots;
}

// out[x] = sum_y kd[|x - y|] v[y] over |x - y| < window (kd is zero beyond: FP64 underflow)
__global__ void k_kernel_conv(const double* __restrict__ v, const double* __restrict__ kd, int64_t dim, int64_t window,
                              double* __restrict__ out) {
  const int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= dim) return;
  const int64_t y0 = x - window + 1 > 0 ? x - window + 1 : 0;
  const int64_t y1 = x + window < dim ? x + window : dim;
  double acc = 0.0;
  for (int64_t y = y0; y < y1; ++y) acc = fma(kd[x > y ? x - y : y - x], v[y], acc);
  out[x] = acc;
}

// dots[k] = sum_x (a_k[x] - b_k[x]) w[x], a_k = dist[2k], b_k = dist[2k+1]; one CTA per k, fixed tree
__global__ void __launch_bounds__(256) k_shift_dots(const double* __restrict__ dist, uint64_t dim,
                                                    const double* __restrict__ w, double* __restrict__ dots) {
  __shared__ double red[256];
  const int k = blockIdx.x;
  const double* a = dist + (size_t)(2 * k) * dim;
  const double* b = a + dim;
  double acc = 0.0;
  for (uint64_t x = threadIdx.x; x < dim; x += 256) acc += (a[x] - b[x]) * w[x];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int h = 128; h > 0; h >>= 1) {
    if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) dots[k] = red[0];
}

// out[0] = sum_x a[x] w[x] (one CTA, fixed tree)
__global__ void __launch_bounds__(256) k_dot(const double* __restrict__ a, const double* __restrict__ w, uint64_t dim,
                                             double* __restrict__ out) {
  __shared__ double red[256];
  double acc = 0.0;
  for (uint64_t x = threadIdx.x; x < dim; x += 256) acc += a[x] * w[x];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int h = 128; h > 0; h >>= 1) {
    if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = red[0];
}

__global__ void k_sub(const double* __restrict__ a, const double* __restrict__ b, uint64_t dim, double* __restrict__ out) {
  const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < dim) out[i] = a[i] - b[i];
}

}  // namespace

}  // namespace qs

using namespace qs;

extern "C" {

int qs_mmd_gradient(const qs_circuit* c, const double* params, const double* host_target, double sigma, int dtype,
                    int nshots, const double* host_u, void* dev_states, void* stream, double* host_grad,
                    double* host_loss) {
  if (!c || !host_target || !host_grad || !dev_states) return fail(QS_EINVAL, "null argument");
  if (!(sigma > 0)) return fail(QS_EINVAL, "sigma must be > 0");
  const int P = c->nparams, n = c->nqubits;
  if (n > 16) return fail(QS_EUNSUPPORTED, "the MMD kernel sums are built for n <= 16");
  if (P > 0 && !params) return fail(QS_EINVAL, "params is NULL");
  if (nshots > 0 && !host_u) return fail(QS_EINVAL, "uniforms are NULL");
  std::vector<int> uses(std::max(1, P), 0);
  for (const qs_gate_desc& g : c->gates) {
    if (g.param < 0) continue;
    const bool pauli_rot = g.kind == QS_GATE_RX || g.kind == QS_GATE_RY || g.kind == QS_GATE_RZ || g.kind == QS_GATE_ROT;
    if (!pauli_rot || g.ctrl_mask) return fail(QS_EUNSUPPORTED, "parameter shift needs uncontrolled Pauli rotations");
    ++uses[g.param];
  }
  for (int k = 0; k < P; ++k)
    if (uses[k] != 1) return fail(QS_EUNSUPPORTED, "parameter %d is used %d times (shift rule needs one use)", k, uses[k]);
  const int R = 2 * P + 1;  // 2k: +pi/2, 2k+1: -pi/2, 2P: unshifted
  const uint64_t dim = 1ull << n;
  cudaStream_t st = (cudaStream_t)stream;
  qs_state* s = nullptr;
  QS_TRY(qs_state_create(n, dtype, R, dev_states, stream, &s));
  std::vector<double> pm((size_t)R * std::max(1, P), 0.0);
  for (int r = 0; r < R; ++r)
    for (int j = 0; j < P; ++j) {
      const int k = r / 2;
      const double sh = (r < 2 * P && j == k) ? ((r & 1) ? -M_PI / 2 : M_PI / 2) : 0.0;
      pm[(size_t)r * P + j] = params[j] + sh;
    }
  int rc = qs_state_reset(s, nullptr);
  if (rc == QS_OK && P > 0) rc = qs_apply_circuit(s, c, pm.data(), QS_APPLY_PER_REGISTER);
  else if (rc == QS_OK) rc = qs_apply_circuit(s, c, nullptr, 0);
  // device scratch: distributions R x dim, target, kd, Kp - Kq, Kq, diff, dots, samples, uniforms
  const size_t nsr = (size_t)R * std::max(1, nshots);
  const size_t sscr = sample_scratch_doubles(n);
  const size_t doubles = (size_t)R * dim + 5 * dim + (size_t)R + 4 + nsr + sscr;
  if (rc == QS_OK) rc = ensure_ws(s, s->ws, sizeof(double) * doubles + sizeof(int64_t) * nsr + 256);
  if (rc != QS_OK) {
    qs_state_destroy(s);
    return rc;
  }
  double* dist = (double*)s->ws.ptr;
  double* dq = dist + (size_t)R * dim;
  double* dkd = dq + dim;
  double* dkp = dkd + dim;  // K p
  double* dkq = dkp + dim;  // K q
  double* dw = dkq + dim;   // K p - K q
  double* ddots = dw + dim;
  double* dsc = ddots + R;  // [0]: p K p, [1]: p K q, [2]: q K q
  double* du = dsc + 4;
  double* dscr = du + nsr;
  int64_t* dsamp = (int64_t*)(dscr + sscr);
  const unsigned gb = (unsigned)((R * dim + 255) / 256), g1 = (unsigned)((dim + 255) / 256);
  auto run = [&]() -> int {
    if (nshots > 0) {
      QS_CUDA(cudaMemsetAsync(dist, 0, sizeof(double) * R * dim, st));
      QS_CUDA(cudaMemcpyAsync(du, host_u, sizeof(double) * nsr, cudaMemcpyHostToDevice, st));
      const size_t ab = amp_bytes(dtype);
      for (int r = 0; r < R; ++r)
        QS_TRY(sample_dev((const char*)s->data + ab * s->off[r], dtype, n, du + (size_t)r * nshots, nshots,
                          dsamp + (size_t)r * nshots, dscr, st));
      k_hist<<<(unsigned)((nsr + 255) / 256), 256, 0, st>>>(dsamp, nshots, R, dim, (unsigned long long*)dist);
      k_counts_to_dist<<<gb, 256, 0, st>>>(dist, (uint64_t)R * dim, nshots);
    } else if (dtype == QS_C64) {
      k_probs<float2><<<gb, 256, 0, st>>>((const float2*)s->data, (uint64_t)R * dim, dist);
    } else {
      k_probs<double2><<<gb, 256, 0, st>>>((const double2*)s->data, (uint64_t)R * dim, dist);
    }
    QS_LAUNCHED();
    // kernel profile kd[d] = exp(-d^2 / (2 sigma^2)), zero where it underflows
    std::vector<double> kd(dim, 0.0);
    int64_t window = 0;
    for (uint64_t d = 0; d < dim; ++d) {
      const double v = std::exp(-(double)d * (double)d / (2.0 * sigma * sigma));
      if (v == 0.0) break;
      kd[d] = v;
      window = (int64_t)d + 1;
    }
    QS_CUDA(cudaMemcpyAsync(dkd, kd.data(), sizeof(double) * dim, cudaMemcpyHostToDevice, st));
    QS_CUDA(cudaMemcpyAsync(dq, host_target, sizeof(double) * dim, cudaMemcpyHostToDevice, st));
    const double* p = dist + (size_t)(2 * P) * dim;
    k_kernel_conv<<<g1, 256, 0, st>>>(p, dkd, (int64_t)dim, window, dkp);
    k_kernel_conv<<<g1, 256, 0, st>>>(dq, dkd, (int64_t)dim, window, dkq);
    k_sub<<<g1, 256, 0, st>>>(dkp, dkq, dim, dw);
    QS_LAUNCHED();
    if (P > 0) k_shift_dots<<<P, 256, 0, st>>>(dist, dim, dw, ddots);
    k_dot<<<1, 256, 0, st>>>(p, dkp, dim, dsc + 0);
    k_dot<<<1, 256, 0, st>>>(p, dkq, dim, dsc + 1);
    k_dot<<<1, 256, 0, st>>>(dq, dkq, dim, dsc + 2);
    QS_LAUNCHED();
    std::vector<double> dots(std::max(1, P)), sc(3);
    if (P > 0) QS_CUDA(cudaMemcpyAsync(dots.data(), ddots, sizeof(double) * P, cudaMemcpyDeviceToHost, st));
    QS_CUDA(cudaMemcpyAsync(sc.data(), dsc, sizeof(double) * 3, cudaMemcpyDeviceToHost, st));
    QS_CUDA(cudaStreamSynchronize(st));
    for (int k = 0; k < P; ++k) host_grad[k] = dots[k];
    if (host_loss) *host_loss = sc[0] - 2.0 * sc[1] + sc[2];
    return QS_OK;
  };
  rc = run();
  qs_state_destroy(s);
  return rc;
}


int qs_observable_groups(const qs_observable* o, int* ngroups) {
  if (!o || !ngroups) return fail(QS_EINVAL, "null argument");
  std::vector<BasisGroup> gs;
  double c = 0;
  group_terms(o, gs, &c);
  *ngroups = (int)gs.size();
  return QS_OK;
}

int qs_shot_expect(qs_state* s, const qs_observable* o, const double* host_u, int nshots, void* dev_work,
                   double* host_out) {
  if (!s || !o || !host_out) return fail(QS_EINVAL, "null argument");
  return shot_expect(s, o, host_u, nshots, dev_work, host_out);
}

int qs_faithful_gradient(const qs_circuit* c, const double* params, const qs_observable* o, int dtype, int nshots,
                         const double* host_u, void* dev_states, void* dev_work, void* stream, double* host_grad) {
  if (!c || !o || !host_grad || !dev_states) return fail(QS_EINVAL, "null argument");
  const int P = c->nparams;
  if (P < 1) return QS_OK;
  if (!params) return fail(QS_EINVAL, "params is NULL");
  // every parameter: exactly one uncontrolled Pauli rotation
  std::vector<int> uses(P, 0);
  for (const qs_gate_desc& g : c->gates) {
    if (g.param < 0) continue;
    const bool pauli_rot = g.kind == QS_GATE_RX || g.kind == QS_GATE_RY || g.kind == QS_GATE_RZ || g.kind == QS_GATE_ROT;
    if (!pauli_rot || g.ctrl_mask) return fail(QS_EUNSUPPORTED, "parameter shift needs uncontrolled Pauli rotations");
    ++uses[g.param];
  }
  for (int k = 0; k < P; ++k)
    if (uses[k] != 1) return fail(QS_EUNSUPPORTED, "parameter %d is used %d times (shift rule needs one use)", k, uses[k]);
  const int R = 2 * P, n = c->nqubits;
  qs_state* st = nullptr;
  QS_TRY(qs_state_create(n, dtype, R, dev_states, stream, &st));
  std::vector<double> pm((size_t)R * P);
  for (int k = 0; k < P; ++k)
    for (int j = 0; j < P; ++j) {
      pm[(size_t)(2 * k) * P + j] = params[j] + (j == k ? M_PI / 2 : 0.0);
      pm[(size_t)(2 * k + 1) * P + j] = params[j] - (j == k ? M_PI / 2 : 0.0);
    }
  int rc = QS_OK;
  bool done = false;
  if (dtype == QS_C64 && n >= 5) {
    // one persistent launch for all 2P registers when the circuit fits the batched engine
    std::vector<const qs_circuit*> cs(R, c);
    qs_observable empty;
    std::vector<const qs_observable*> os(R, &empty);
    qs_batch_program* prog = nullptr;
    if (qs_batch_program_create(R, cs.data(), os.data(), 0, &prog) == QS_OK) {
      double* dparams = nullptr;
      if (cudaMalloc(&dparams, sizeof(double) * (pm.size() + R)) == cudaSuccess) {
        rc = qs_state_reset(st, nullptr);
        if (rc == QS_OK && cudaMemcpyAsync(dparams, pm.data(), sizeof(double) * pm.size(), cudaMemcpyHostToDevice,
                                           (cudaStream_t)stream) != cudaSuccess)
          rc = fail(QS_EDEVICE, "parameter upload failed");
        if (rc == QS_OK) rc = qs_batch_run(st, prog, dparams, dparams + pm.size(), nullptr, QS_BATCH_RESET);
        if (rc == QS_OK) rc = qs_state_sync(st);
        cudaFree(dparams);
        done = rc == QS_OK;
      } else {
        cudaGetLastError();
      }
      qs_batch_program_destroy(prog);
    }
  }
  if (!done && rc == QS_OK) {
    rc = qs_state_reset(st, nullptr);
    if (rc == QS_OK) rc = qs_apply_circuit(st, c, pm.data(), QS_APPLY_PER_REGISTER);
  }
  std::vector<double> E(R, 0.0);
  if (rc == QS_OK) rc = nshots > 0 ? shot_expect(st, o, host_u, nshots, dev_work, E.data()) : qs_expect(st, o, E.data());
  qs_state_destroy(st);
  if (rc != QS_OK) return rc;
  for (int k = 0; k < P; ++k) host_grad[k] = 0.5 * (E[2 * k] - E[2 * k + 1]);
  return QS_OK;
}

}  // extern "C"
