// sparse.cu -- sparse (CSR) matrix of a sum of Pauli strings, the matrix
// representation of a Hamiltonian block (Sec. "Matrix Representation";
// App. "Matrix Types": sums of Pauli strings are sparse; benchmarked in
// Sec. "Matrix Representation and AD Performance" as mat(heisenberg(20))).
//
// A term c P with P = i^{popcount(x&z)} X^x Z^z (the convention of qs_expect)
// maps |j> to c i^{popcount(x&z)} (-1)^{popcount(j&z)} |j ^ x>.  Row i of the
// matrix therefore has one candidate column j = i ^ x per distinct x among the
// terms, with value sum over the terms t with x_t = x of
// c_t i^{popcount(x_t & z_t)} (-1)^{popcount(j & z_t)}.  Entries that sum to
// exactly zero are dropped; columns are ascending within a row.
//
// Three launches: per-row nonzero counts, an exclusive scan of the counts
// into row pointers (per-block scans, a scan of the block totals, offsets
// added), and a fill pass that recomputes each row's entries and writes them
// in column order.
#include <algorithm>
#include <cstring>

#include "common.cuh"

namespace qs {

namespace {

constexpr int kSpMaxGroups = 64;   // distinct x masks (entries per row at most)
constexpr int kSpMaxTerms = 256;
constexpr int kScanThreads = 1024;

struct SpTerms {
  int ngroups;
  uint64_t xm[kSpMaxGroups];       // distinct x masks
  int t0[kSpMaxGroups + 1];        // terms of group g: t0[g] .. t0[g+1]-1
  uint64_t z[kSpMaxTerms];
  double cre[kSpMaxTerms], cim[kSpMaxTerms];  // c i^{popcount(x&z)}
};

__device__ __forceinline__ double2 entry(const SpTerms& T, int g, uint64_t j) {
  double re = 0.0, im = 0.0;
  for (int t = T.t0[g]; t < T.t0[g + 1]; ++t) {
    const double s = (__popcll(j & T.z[t]) & 1) ? -1.0 : 1.0;
    re += s * T.cre[t];
    im += s * T.cim[t];
  }
  return make_double2(re, im);
}

__global__ void k_sp_count(const __grid_constant__ SpTerms T, uint64_t dim, int64_t* __restrict__ counts) {
  const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= dim) return;
  int c = 0;
  for (int g = 0; g < T.ngroups; ++g) {
    const double2 v = entry(T, g, i ^ T.xm[g]);
    c += (v.x != 0.0 || v.y != 0.0);
  }
  counts[i] = c;
}

// exclusive scan of one block of kScanThreads counts in place; block total to sums[block]
__global__ void __launch_bounds__(kScanThreads) k_scan_block(int64_t* __restrict__ a, uint64_t n,
                                                             int64_t* __restrict__ sums) {
  __shared__ int64_t s[kScanThreads];
  const uint64_t i = (uint64_t)blockIdx.x * kScanThreads + threadIdx.x;
  s[threadIdx.x] = i < n ? a[i] : 0;
  __syncthreads();
  for (int off = 1; off < kScanThreads; off <<= 1) {  // inclusive Hillis-Steele
    const int64_t v = threadIdx.x >= (unsigned)off ? s[threadIdx.x - off] : 0;
    __syncthreads();
    s[threadIdx.x] += v;
    __syncthreads();
  }
  if (i < n) a[i] = threadIdx.x ? s[threadIdx.x - 1] : 0;
  if (threadIdx.x == kScanThreads - 1) sums[blockIdx.x] = s[kScanThreads - 1];
}

// exclusive scan of the block totals (one thread, in order) and the grand total at sums[nb]
__global__ void k_scan_sums(int64_t* __restrict__ sums, uint64_t nb) {
  int64_t acc = 0;
  for (uint64_t b = 0; b < nb; ++b) {
    const int64_t v = sums[b];
    sums[b] = acc;
    acc += v;
  }
  sums[nb] = acc;
}

__global__ void k_scan_add(int64_t* __restrict__ a, uint64_t n, const int64_t* __restrict__ sums) {
  const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) a[i] += sums[i / kScanThreads];
  if (i == n - 1) a[n] = sums[(n + kScanThreads - 1) / kScanThreads];
}

__global__ void k_sp_fill(const __grid_constant__ SpTerms T, uint64_t dim, const int64_t* __restrict__ rowptr,
                          int64_t* __restrict__ cols, double2* __restrict__ vals) {
  const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= dim) return;
  int64_t w = rowptr[i];
  // emit in ascending column order: repeatedly take the smallest column above the last one
  uint64_t last = 0;
  bool first = true;
  for (int k = 0; k < T.ngroups; ++k) {
    int best = -1;
    uint64_t bj = 0;
    for (int g = 0; g < T.ngroups; ++g) {
      const uint64_t j = i ^ T.xm[g];
      if ((first || j > last) && (best < 0 || j < bj)) {
        best = g;
        bj = j;
      }
    }
    if (best < 0) break;
    first = false;
    last = bj;
    const double2 v = entry(T, best, bj);
    if (v.x != 0.0 || v.y != 0.0) {
      cols[w] = (int64_t)bj;
      vals[w] = v;
      ++w;
    }
  }
}

int build_terms(const qs_observable* o, int n, SpTerms* T) {
  std::memset(T, 0, sizeof(*T));
  std::vector<uint64_t> xs;
  for (const qs_pauli_term& p : o->terms) {
    if (n < 64 && ((p.x_mask | p.z_mask) >> n)) return fail(QS_EINVAL, "a term acts beyond qubit %d", n - 1);
    if (std::find(xs.begin(), xs.end(), p.x_mask) == xs.end()) xs.push_back(p.x_mask);
  }
  if ((int)xs.size() > kSpMaxGroups) return fail(QS_EUNSUPPORTED, "more than %d distinct X patterns", kSpMaxGroups);
  if ((int)o->terms.size() > kSpMaxTerms) return fail(QS_EUNSUPPORTED, "more than %d terms", kSpMaxTerms);
  T->ngroups = (int)xs.size();
  int t = 0;
  for (int g = 0; g < T->ngroups; ++g) {
    T->xm[g] = xs[g];
    T->t0[g] = t;
    for (const qs_pauli_term& p : o->terms) {
      if (p.x_mask != xs[g]) continue;
      T->z[t] = p.z_mask;
      // c * i^{popcount(x & z)}
      const int ny = __builtin_popcountll(p.x_mask & p.z_mask) & 3;
      const double re[4] = {1, 0, -1, 0}, im[4] = {0, 1, 0, -1};
      T->cre[t] = p.coeff * re[ny];
      T->cim[t] = p.coeff * im[ny];
      ++t;
    }
  }
  T->t0[T->ngroups] = t;
  return QS_OK;
}

}  // namespace

}  // namespace qs

using namespace qs;

extern "C" {

int qs_observable_csr_rows(const qs_observable* o, int nqubits, int64_t* dev_rowptr, int64_t* dev_scratch,
                           int64_t* host_nnz, void* stream) {
  if (!o || !dev_rowptr || !dev_scratch || !host_nnz) return fail(QS_EINVAL, "null argument");
  if (nqubits < 1 || nqubits > 34) return fail(QS_EINVAL, "nqubits must be in 1..34");
  SpTerms T;
  QS_TRY(build_terms(o, nqubits, &T));
  cudaStream_t st = (cudaStream_t)stream;
  const uint64_t dim = 1ull << nqubits, nb = (dim + kScanThreads - 1) / kScanThreads;
  k_sp_count<<<(unsigned)((dim + 255) / 256), 256, 0, st>>>(T, dim, dev_rowptr);
  QS_LAUNCHED();
  k_scan_block<<<(unsigned)nb, kScanThreads, 0, st>>>(dev_rowptr, dim, dev_scratch);
  QS_LAUNCHED();
  k_scan_sums<<<1, 1, 0, st>>>(dev_scratch, nb);
  QS_LAUNCHED();
  k_scan_add<<<(unsigned)((dim + 255) / 256), 256, 0, st>>>(dev_rowptr, dim, dev_scratch);
  QS_LAUNCHED();
  QS_CUDA(cudaMemcpyAsync(host_nnz, dev_rowptr + dim, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
  QS_CUDA(cudaStreamSynchronize(st));
  return QS_OK;
}

int qs_observable_csr_fill(const qs_observable* o, int nqubits, const int64_t* dev_rowptr, int64_t* dev_cols,
                           double* dev_vals, void* stream) {
  if (!o || !dev_rowptr || !dev_cols || !dev_vals) return fail(QS_EINVAL, "null argument");
  if (nqubits < 1 || nqubits > 34) return fail(QS_EINVAL, "nqubits must be in 1..34");
  SpTerms T;
  QS_TRY(build_terms(o, nqubits, &T));
  cudaStream_t st = (cudaStream_t)stream;
  const uint64_t dim = 1ull << nqubits;
  k_sp_fill<<<(unsigned)((dim + 255) / 256), 256, 0, st>>>(T, dim, dev_rowptr, dev_cols, (double2*)dev_vals);
  QS_LAUNCHED();
  return QS_OK;
}

}  // extern "C"
