// vecops.cu -- level-1 operations between two states of the same shape
// (copy, inner product, y += alpha x) and the host-side gate matrices of a
// circuit's gates.  They are the pieces a caller needs to run the reversible
// adjoint of Sec. "Reverse Mode" gate by gate over a state that is split into
// pieces (for instance across processes): the gradient of a parameterised gate
// is 2 c Im<lambda|H|psi> (Eq. apply-back, U = exp(-i theta c H)), an inner
// product of lambda with H psi, and lambda = O psi is a sum of Pauli strings
// applied to copies of psi.
//
// Inner products accumulate in FP64 (products of the stored amplitudes widened
// to FP64), per-block partials are folded in block order, so the result does
// not depend on scheduling.
#include <algorithm>
#include <cstring>

#include "common.cuh"

namespace qs {

constexpr int kVecThreads = 256;
constexpr int kVecMaxBlocks = 1216;  // 8 per SM

__device__ __forceinline__ double2 wide(float2 v) { return make_double2((double)v.x, (double)v.y); }
__device__ __forceinline__ double2 wide(double2 v) { return v; }

// partials[(r * nblk + block) * 2 + {0, 1}] = Re, Im of sum conj(a_i) b_i over the block's share
template <typename T>
__global__ void __launch_bounds__(kVecThreads)
k_inner(const T* __restrict__ a, const T* __restrict__ b, const int64_t* __restrict__ off, double* __restrict__ partials) {
  const int nblk = gridDim.x;
  const int64_t r = blockIdx.y;
  const int64_t base = off[r], len = off[r + 1] - off[r];
  double re = 0.0, im = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * kVecThreads + threadIdx.x; i < len; i += (int64_t)nblk * kVecThreads) {
    const double2 x = wide(a[base + i]), y = wide(b[base + i]);
    re += x.x * y.x + x.y * y.y;
    im += x.x * y.y - x.y * y.x;
  }
  __shared__ double red[2][kVecThreads / 32];
  for (int o = 16; o > 0; o >>= 1) {
    re += __shfl_xor_sync(0xffffffffu, re, o);
    im += __shfl_xor_sync(0xffffffffu, im, o);
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) { red[0][warp] = re; red[1][warp] = im; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double sr = 0.0, si = 0.0;
    for (int w = 0; w < kVecThreads / 32; ++w) { sr += red[0][w]; si += red[1][w]; }
    partials[(r * nblk + blockIdx.x) * 2] = sr;
    partials[(r * nblk + blockIdx.x) * 2 + 1] = si;
  }
}

__global__ void k_inner_final(const double* __restrict__ partials, int nblk, int nreg, double* __restrict__ out) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nreg) return;
  double sr = 0.0, si = 0.0;
  for (int b = 0; b < nblk; ++b) {
    sr += partials[((size_t)r * nblk + b) * 2];
    si += partials[((size_t)r * nblk + b) * 2 + 1];
  }
  out[2 * r] = sr;
  out[2 * r + 1] = si;
}

// y_i += alpha x_i in the state's precision
template <typename T>
__global__ void __launch_bounds__(kVecThreads)
k_axpy(T* __restrict__ y, const T* __restrict__ x, uint64_t total, T alpha) {
  for (uint64_t i = (uint64_t)blockIdx.x * kVecThreads + threadIdx.x; i < total;
       i += (uint64_t)gridDim.x * kVecThreads) {
    const T v = x[i];
    T w = y[i];
    w.x = fma(alpha.x, v.x, fma(-alpha.y, v.y, w.x));
    w.y = fma(alpha.x, v.y, fma(alpha.y, v.x, w.y));
    y[i] = w;
  }
}

template <typename S, typename D>
__global__ void __launch_bounds__(kVecThreads) k_convert(const S* __restrict__ in, D* __restrict__ out, uint64_t total) {
  for (uint64_t i = (uint64_t)blockIdx.x * kVecThreads + threadIdx.x; i < total; i += (uint64_t)gridDim.x * kVecThreads) {
    const S v = in[i];
    D w;
    w.x = v.x;
    w.y = v.y;
    out[i] = w;
  }
}

static int same_shape(const qs_state* a, const qs_state* b) {
  if (!a || !b) return fail(QS_EINVAL, "null state");
  if (a->dtype != b->dtype) return fail(QS_EINVAL, "states differ in dtype");
  if (a->nq != b->nq) return fail(QS_EINVAL, "states differ in register sizes");
  return QS_OK;
}

}  // namespace qs

using namespace qs;

extern "C" {

int qs_state_copy(qs_state* dst, const qs_state* src) {
  if (dst && src && dst->dtype != src->dtype && dst->nq == src->nq) {
    // complex64 <-> complex128: widened exactly, or rounded to nearest
    const uint64_t total = (uint64_t)dst->off.back();
    const unsigned grid = (unsigned)std::max<uint64_t>(1, std::min<uint64_t>((total + kVecThreads - 1) / kVecThreads,
                                                                           (uint64_t)kVecMaxBlocks * 4));
    if (dst->dtype == QS_C128)
      k_convert<float2, double2><<<grid, kVecThreads, 0, dst->stream>>>((const float2*)src->data, (double2*)dst->data, total);
    else
      k_convert<double2, float2><<<grid, kVecThreads, 0, dst->stream>>>((const double2*)src->data, (float2*)dst->data, total);
    QS_LAUNCHED();
    return QS_OK;
  }
  QS_TRY(same_shape(dst, src));
  if (dst->data == src->data) return QS_OK;
  QS_CUDA(cudaMemcpyAsync(dst->data, src->data, (size_t)dst->off.back() * amp_bytes(dst->dtype),
                          cudaMemcpyDeviceToDevice, dst->stream));
  return QS_OK;
}

int qs_state_inner(qs_state* a, const qs_state* b, double* host_out) {
  QS_TRY(same_shape(a, b));
  if (!host_out) return fail(QS_EINVAL, "null output");
  cudaStream_t st = a->stream;
  const int nreg = a->nreg;
  int64_t maxlen = 0;
  for (int r = 0; r < nreg; ++r) maxlen = std::max<int64_t>(maxlen, a->off[r + 1] - a->off[r]);
  const int nblk = (int)std::max<int64_t>(
      1, std::min<int64_t>(maxlen / (kVecThreads * 8), std::max(1, kVecMaxBlocks / std::max(1, nreg))));
  const size_t off_bytes = sizeof(int64_t) * (nreg + 1);
  const size_t part_off = (off_bytes + 255) / 256 * 256;
  const size_t out_off = part_off + (sizeof(double) * 2 * (size_t)nreg * nblk + 255) / 256 * 256;
  QS_TRY(ensure_ws(a, a->ws, out_off + sizeof(double) * 2 * nreg));
  int64_t* doff = (int64_t*)a->ws.ptr;
  double* partials = (double*)((char*)a->ws.ptr + part_off);
  double* dout = (double*)((char*)a->ws.ptr + out_off);
  QS_CUDA(cudaMemcpyAsync(doff, a->off.data(), off_bytes, cudaMemcpyHostToDevice, st));
  dim3 grid(nblk, nreg);
  if (a->dtype == QS_C64)
    k_inner<float2><<<grid, kVecThreads, 0, st>>>((const float2*)a->data, (const float2*)b->data, doff, partials);
  else
    k_inner<double2><<<grid, kVecThreads, 0, st>>>((const double2*)a->data, (const double2*)b->data, doff, partials);
  QS_LAUNCHED();
  k_inner_final<<<(nreg + 127) / 128, 128, 0, st>>>(partials, nblk, nreg, dout);
  QS_LAUNCHED();
  QS_CUDA(cudaMemcpyAsync(host_out, dout, sizeof(double) * 2 * nreg, cudaMemcpyDeviceToHost, st));
  QS_CUDA(cudaStreamSynchronize(st));
  return QS_OK;
}

int qs_state_axpy(qs_state* y, double alpha_re, double alpha_im, const qs_state* x) {
  QS_TRY(same_shape(y, x));
  if (y->data == x->data) return fail(QS_EINVAL, "x and y must be distinct buffers");
  const uint64_t total = (uint64_t)y->off.back();
  const unsigned grid = (unsigned)std::max<uint64_t>(1, std::min<uint64_t>((total + kVecThreads - 1) / kVecThreads,
                                                                         (uint64_t)kVecMaxBlocks * 4));
  if (y->dtype == QS_C64)
    k_axpy<float2><<<grid, kVecThreads, 0, y->stream>>>((float2*)y->data, (const float2*)x->data, total,
                                                         make_float2((float)alpha_re, (float)alpha_im));
  else
    k_axpy<double2><<<grid, kVecThreads, 0, y->stream>>>((double2*)y->data, (const double2*)x->data, total,
                                                          make_double2(alpha_re, alpha_im));
  QS_LAUNCHED();
  return QS_OK;
}

int qs_circuit_gate_matrices(const qs_circuit* c, int index, const double* host_params, qs_gate_desc* host_desc,
                             double* host_U, double* host_G, double* host_cfac) {
  if (!c) return fail(QS_EINVAL, "null circuit");
  if (index < 0 || index >= (int)c->gates.size()) return fail(QS_EINVAL, "gate index %d out of range", index);
  const qs_gate_desc& g = c->gates[index];
  if (g.param >= 0 && !host_params) return fail(QS_EINVAL, "gate %d needs the parameter vector", index);
  if (host_desc) *host_desc = g;
  const int D = 1 << g.nlocs;
  if (host_U) {
    std::vector<cd> U;
    QS_TRY(gate_matrix(c, g, host_params, U));
    for (int i = 0; i < D * D; ++i) { host_U[2 * i] = U[i].real(); host_U[2 * i + 1] = U[i].imag(); }
  }
  if (host_G || host_cfac) {
    if (g.param < 0) return fail(QS_EINVAL, "gate %d has no parameter", index);
    std::vector<cd> G;
    double cf = 0.0;
    QS_TRY(gate_generator(g, G, &cf));
    if (host_G)
      for (int i = 0; i < D * D; ++i) { host_G[2 * i] = G[i].real(); host_G[2 * i + 1] = G[i].imag(); }
    if (host_cfac) *host_cfac = cf;
  }
  return QS_OK;
}

}  // extern "C"
