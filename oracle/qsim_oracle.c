/*
 * qsim_oracle.c -- plain, slow FP64 state-vector simulator.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, the smoke check and the bench's CPU
 * baseline may load this library.  It shares no code, header, table or helper
 * with the CUDA path; every routine restates a definition from the paper
 * (Yao.jl, arXiv 1912.10877) as directly as possible, with no fusion, no
 * blocking and no specialisation beyond that definition.
 *
 * Conventions (Sec. "Instructions on Quantum Registers"): little-endian, qubit
 * loc l is bit l of the basis index; a k-qubit gate on locs (l_0..l_{k-1}) has
 * matrix index bit j <-> qubit l_j.  Control value 1 = control, 0 = inverse
 * control.
 *
 * Build: gcc -O2 -std=c11 -fPIC -shared -fopenmp -ffp-contract=off
 * (-ffp-contract=off keeps |a|^2 = re*re + im*im a separately rounded multiply
 * and add, which the measurement contract below relies on).
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;

#define ORC_MAXK 5
#define ORC_MAXC 16
#define ORC_MAXOPS 64

/* gate kinds, private to the oracle (the Python wrapper maps names to these) */
enum {
  ORC_I = 0, ORC_X, ORC_Y, ORC_Z, ORC_H, ORC_S, ORC_SDG, ORC_T, ORC_TDG,
  ORC_RX, ORC_RY, ORC_RZ, ORC_SHIFT, ORC_PHASE, ORC_SWAP, ORC_ROT, ORC_MATRIX
};

typedef struct {
  int32_t kind;
  int32_t k;                    /* number of targets */
  int32_t locs[ORC_MAXK];
  int32_t nctrl;
  int32_t ctrl_locs[ORC_MAXC];
  int32_t ctrl_vals[ORC_MAXC];
  int32_t param;                /* -1: fixed angle */
  int32_t paulis[ORC_MAXK];     /* ROT: 1 = X, 2 = Y, 3 = Z per target */
  int64_t mat_offset;           /* MATRIX: offset (complex entries) into the matrix pool */
  double theta;                 /* fixed angle when param < 0 */
} orc_gate;

typedef struct {
  double coeff;
  int32_t nops;
  int32_t locs[ORC_MAXOPS];
  int32_t paulis[ORC_MAXOPS];   /* 1 = X, 2 = Y, 3 = Z */
} orc_term;

/* ------------------------------------------------------------------------ */
/* Pauli matrices and gate matrices (paper App. "Builtin Block Types";       */
/* rotations R_S(theta) = exp(-i S theta / 2), Sec. "Forward Mode";          */
/* shift(theta) = diag(1, e^{i theta}), listing "inspecting gates").         */
/* ------------------------------------------------------------------------ */

static void pauli2(int p, cplx m[2][2]) {
  m[0][0] = m[0][1] = m[1][0] = m[1][1] = 0;
  if (p == 0) { m[0][0] = 1; m[1][1] = 1; }
  if (p == 1) { m[0][1] = 1; m[1][0] = 1; }
  if (p == 2) { m[0][1] = -I; m[1][0] = I; }
  if (p == 3) { m[0][0] = 1; m[1][1] = -1; }
}

/* U (row-major, 2^k x 2^k) of gate g at angle theta */
int orc_gate_matrix(const orc_gate* g, double theta, const cplx* mats, cplx* U) {
  int k = g->k;
  int K = 1 << k;
  memset(U, 0, sizeof(cplx) * K * K);
  double c = cos(theta / 2), s = sin(theta / 2);
  switch (g->kind) {
    case ORC_I: U[0] = 1; U[3] = 1; break;
    case ORC_X: U[1] = 1; U[2] = 1; break;
    case ORC_Y: U[1] = -I; U[2] = I; break;
    case ORC_Z: U[0] = 1; U[3] = -1; break;
    case ORC_H: U[0] = U[1] = U[2] = 1 / sqrt(2.0); U[3] = -1 / sqrt(2.0); break;
    case ORC_S: U[0] = 1; U[3] = I; break;
    case ORC_SDG: U[0] = 1; U[3] = -I; break;
    case ORC_T: U[0] = 1; U[3] = cexp(I * M_PI / 4); break;
    case ORC_TDG: U[0] = 1; U[3] = cexp(-I * M_PI / 4); break;
    case ORC_RX: U[0] = c; U[1] = -I * s; U[2] = -I * s; U[3] = c; break;
    case ORC_RY: U[0] = c; U[1] = -s; U[2] = s; U[3] = c; break;
    case ORC_RZ: U[0] = cexp(-I * theta / 2); U[3] = cexp(I * theta / 2); break;
    case ORC_SHIFT: U[0] = 1; U[3] = cexp(I * theta); break;
    case ORC_PHASE: U[0] = cexp(I * theta); U[3] = cexp(I * theta); break;
    case ORC_SWAP: /* |b0 b1> -> |b1 b0>: index 1 <-> 2 */
      U[0 * 4 + 0] = 1; U[1 * 4 + 2] = 1; U[2 * 4 + 1] = 1; U[3 * 4 + 3] = 1; break;
    case ORC_ROT: { /* cos(theta/2) 1 - i sin(theta/2) (sigma_{p_0} (x) ... ), bit j <-> target j */
      for (int r = 0; r < K; ++r)
        for (int col = 0; col < K; ++col) {
          cplx prod = 1;
          for (int j = 0; j < k; ++j) {
            cplx m[2][2];
            pauli2(g->paulis[j], m);
            prod *= m[(r >> j) & 1][(col >> j) & 1];
          }
          U[r * K + col] = (r == col ? c : 0) - I * s * prod;
        }
      break;
    }
    case ORC_MATRIX: memcpy(U, mats + g->mat_offset, sizeof(cplx) * K * K); break;
    default: return -1;
  }
  return 0;
}

/* Hermitian conjugate by the paper's dagger rules (Sec. "Manipulating Quantum
 * Circuits"): Hermitian gates unchanged, rotations/shift/phase negate the
 * angle, S<->Sdag and T<->Tdag, a general matrix takes its conjugate transpose. */
int orc_gate_matrix_dagger(const orc_gate* g, double theta, const cplx* mats, cplx* U) {
  orc_gate d = *g;
  switch (g->kind) {
    case ORC_I: case ORC_X: case ORC_Y: case ORC_Z: case ORC_H: case ORC_SWAP:
      return orc_gate_matrix(&d, theta, mats, U);
    case ORC_S: d.kind = ORC_SDG; return orc_gate_matrix(&d, theta, mats, U);
    case ORC_SDG: d.kind = ORC_S; return orc_gate_matrix(&d, theta, mats, U);
    case ORC_T: d.kind = ORC_TDG; return orc_gate_matrix(&d, theta, mats, U);
    case ORC_TDG: d.kind = ORC_T; return orc_gate_matrix(&d, theta, mats, U);
    case ORC_RX: case ORC_RY: case ORC_RZ: case ORC_SHIFT: case ORC_PHASE: case ORC_ROT:
      return orc_gate_matrix(&d, -theta, mats, U);
    case ORC_MATRIX: {
      int K = 1 << g->k;
      const cplx* M = mats + g->mat_offset;
      for (int r = 0; r < K; ++r)
        for (int col = 0; col < K; ++col) U[r * K + col] = conj(M[col * K + r]);
      return 0;
    }
  }
  return -1;
}

/* ------------------------------------------------------------------------ */
/* General multi-control, multi-qubit, arbitrary-location instruction        */
/* (Sec. "Performance", the fallback instruction): for every base index b    */
/* whose target bits are all 0 and whose control bits equal the control      */
/* values, gather the 2^k amplitudes x_m = psi[b + sum_j m_j 2^{l_j}] and    */
/* write back y = U x.                                                       */
/* ------------------------------------------------------------------------ */
void orc_apply(cplx* psi, int n, int k, const int32_t* locs, const cplx* U,
               int nctrl, const int32_t* ctrl_locs, const int32_t* ctrl_vals) {
  int64_t dim = (int64_t)1 << n;
  int K = 1 << k;
  uint64_t locmask = 0;
  for (int j = 0; j < k; ++j) locmask |= 1ull << locs[j];
#pragma omp parallel for schedule(static)
  for (int64_t b = 0; b < dim; ++b) {
    if ((uint64_t)b & locmask) continue;
    int match = 1;
    for (int c = 0; c < nctrl; ++c)
      if ((((uint64_t)b >> ctrl_locs[c]) & 1u) != (uint64_t)ctrl_vals[c]) match = 0;
    if (!match) continue;
    uint64_t idx[1 << ORC_MAXK];
    cplx x[1 << ORC_MAXK], y[1 << ORC_MAXK];
    for (int m = 0; m < K; ++m) {
      uint64_t i = (uint64_t)b;
      for (int j = 0; j < k; ++j)
        if ((m >> j) & 1) i |= 1ull << locs[j];
      idx[m] = i;
      x[m] = psi[i];
    }
    for (int m = 0; m < K; ++m) {
      cplx acc = 0;
      for (int mm = 0; mm < K; ++mm) acc += U[m * K + mm] * x[mm];
      y[m] = acc;
    }
    for (int m = 0; m < K; ++m) psi[idx[m]] = y[m];
  }
}

static double gate_angle(const orc_gate* g, const double* params) {
  return g->param >= 0 ? params[g->param] : g->theta;
}

static int check_gate(const orc_gate* g, int n) {
  if (g->k < 1 || g->k > ORC_MAXK || g->nctrl < 0 || g->nctrl > ORC_MAXC) return -1;
  uint64_t seen = 0;
  for (int j = 0; j < g->k; ++j) {
    if (g->locs[j] < 0 || g->locs[j] >= n || (seen >> g->locs[j]) & 1) return -1;
    seen |= 1ull << g->locs[j];
  }
  for (int c = 0; c < g->nctrl; ++c) {
    if (g->ctrl_locs[c] < 0 || g->ctrl_locs[c] >= n || (seen >> g->ctrl_locs[c]) & 1) return -1;
    seen |= 1ull << g->ctrl_locs[c];
  }
  return 0;
}

/* apply! of a chain: gates in list order (a chain is the matrix product in
 * reverse order, Sec. "Representing Quantum Circuits").  dagger != 0 applies
 * the Hermitian conjugate of the chain: reversed order, each gate daggered. */
int orc_apply_circuit(cplx* psi, int n, const orc_gate* gates, int ngates,
                      const double* params, const cplx* mats, int dagger) {
  cplx U[1 << (2 * ORC_MAXK)];
  for (int t = 0; t < ngates; ++t) {
    const orc_gate* g = &gates[dagger ? ngates - 1 - t : t];
    if (check_gate(g, n)) return -1;
    double th = gate_angle(g, params);
    int rc = dagger ? orc_gate_matrix_dagger(g, th, mats, U) : orc_gate_matrix(g, th, mats, U);
    if (rc) return rc;
    orc_apply(psi, n, g->k, g->locs, U, g->nctrl, g->ctrl_locs, g->ctrl_vals);
  }
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Expectation <psi|O|psi> for O = sum_t c_t P_t, P_t a Pauli string          */
/* (Sec. "Forward Mode", expect).  Each <psi|P_t psi> is summed pairwise       */
/* (recursive halving) in FP64.                                              */
/* ------------------------------------------------------------------------ */
double orc_pairwise_sum(const double* v, int64_t len) {
  if (len <= 0) return 0.0;
  if (len == 1) return v[0];
  int64_t h = len / 2;
  return orc_pairwise_sum(v, h) + orc_pairwise_sum(v + h, len - h);
}

static int check_term(const orc_term* t, int n) {
  if (t->nops < 0 || t->nops > ORC_MAXOPS) return -1;
  uint64_t seen = 0;
  for (int j = 0; j < t->nops; ++j) {
    if (t->locs[j] < 0 || t->locs[j] >= n || (seen >> t->locs[j]) & 1) return -1;
    if (t->paulis[j] < 1 || t->paulis[j] > 3) return -1;
    seen |= 1ull << t->locs[j];
  }
  return 0;
}

/* out = P psi (a fresh copy with each single-qubit Pauli applied) */
static void apply_pauli_string(cplx* out, const cplx* psi, int n, const orc_term* t) {
  int64_t dim = (int64_t)1 << n;
  memcpy(out, psi, sizeof(cplx) * dim);
  for (int j = 0; j < t->nops; ++j) {
    cplx m[2][2];
    pauli2(t->paulis[j], m);
    cplx U[4] = {m[0][0], m[0][1], m[1][0], m[1][1]};
    orc_apply(out, n, 1, &t->locs[j], U, 0, NULL, NULL);
  }
}

int orc_expect(const cplx* psi, int n, const orc_term* terms, int nterms, double* out) {
  int64_t dim = (int64_t)1 << n;
  cplx* phi = malloc(sizeof(cplx) * dim);
  double* prod = malloc(sizeof(double) * dim);
  double* vals = malloc(sizeof(double) * (nterms > 0 ? nterms : 1));
  if (!phi || !prod || !vals) { free(phi); free(prod); free(vals); return -2; }
  int rc = 0;
  for (int t = 0; t < nterms && !rc; ++t) {
    if (check_term(&terms[t], n)) { rc = -1; break; }
    apply_pauli_string(phi, psi, n, &terms[t]);
    for (int64_t i = 0; i < dim; ++i) prod[i] = creal(conj(psi[i]) * phi[i]);
    vals[t] = terms[t].coeff * orc_pairwise_sum(prod, dim);
  }
  if (!rc) *out = orc_pairwise_sum(vals, nterms);
  free(phi); free(prod); free(vals);
  return rc;
}

/* lambda = O psi */
int orc_apply_observable(cplx* lam, const cplx* psi, int n, const orc_term* terms, int nterms) {
  int64_t dim = (int64_t)1 << n;
  cplx* phi = malloc(sizeof(cplx) * dim);
  if (!phi) return -2;
  for (int64_t i = 0; i < dim; ++i) lam[i] = 0;
  for (int t = 0; t < nterms; ++t) {
    if (check_term(&terms[t], n)) { free(phi); return -1; }
    apply_pauli_string(phi, psi, n, &terms[t]);
    for (int64_t i = 0; i < dim; ++i) lam[i] += terms[t].coeff * phi[i];
  }
  free(phi);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Reverse-mode gradient with reversible uncompute (Sec. "Reverse Mode",      */
/* Eqs. apply-back and outer-product).                                       */
/*   forward: psi_{k+1} = U_k psi_k, L = <psi_N|O|psi_N>                     */
/*   adjoint: lambda = dL/dpsi* (Wirtinger), lambda_N = O psi_N              */
/*   backward, k = N-1 .. 0, with psi, lambda the states after gate k:       */
/*     a gate U = exp(-i theta c H) (H Hermitian, including its control      */
/*     projector) contributes dL/dtheta = 2 c Im<lambda|H|psi>;              */
/*     then psi <- U^dag psi, lambda <- U^dag lambda.                        */
/*   Rotations (RX, RY, RZ, ROT): c = 1/2, H = the Pauli (string).           */
/*   shift(theta) = diag(1, e^{i theta}): c = -1, H = P1 on the target.      */
/*   phase(theta) = e^{i theta}: c = -1, H = identity on the target.          */
/* Gradients of shared parameters add up.                                    */
/* ------------------------------------------------------------------------ */
/* One gate of that walk: the contribution of gate g (if it has a parameter)
   to grad, then psi <- U^dag psi and lambda <- U^dag lambda.  phi and im are
   scratch vectors of 2^n entries. */
int orc_adjoint_step(cplx* psi, cplx* lam, cplx* phi, double* im, int n, const orc_gate* g,
                     const double* params, int nparams, const cplx* mats, double* grad) {
  int64_t dim = (int64_t)1 << n;
  int rc = 0;
  cplx U[1 << (2 * ORC_MAXK)];
  {
    double th = gate_angle(g, params);
    if (g->param >= 0) {
      double cfac;
      if (g->param >= nparams) return -1;
      /* phi = H psi, H = (control projector) (x) H_local */
      memcpy(phi, psi, sizeof(cplx) * dim);
      for (int64_t i = 0; i < dim; ++i) {
        int match = 1;
        for (int c = 0; c < g->nctrl; ++c)
          if ((((uint64_t)i >> g->ctrl_locs[c]) & 1u) != (uint64_t)g->ctrl_vals[c]) match = 0;
        if (!match) phi[i] = 0;
      }
      int K = 1 << g->k;
      memset(U, 0, sizeof(cplx) * K * K);
      switch (g->kind) {
        case ORC_RX: U[1] = 1; U[2] = 1; cfac = 0.5; break;
        case ORC_RY: U[1] = -I; U[2] = I; cfac = 0.5; break;
        case ORC_RZ: U[0] = 1; U[3] = -1; cfac = 0.5; break;
        case ORC_ROT:
          for (int r = 0; r < K; ++r)
            for (int col = 0; col < K; ++col) {
              cplx prod = 1;
              for (int j = 0; j < g->k; ++j) {
                cplx m[2][2];
                pauli2(g->paulis[j], m);
                prod *= m[(r >> j) & 1][(col >> j) & 1];
              }
              U[r * K + col] = prod;
            }
          cfac = 0.5;
          break;
        case ORC_SHIFT: U[3] = 1; cfac = -1.0; break;
        case ORC_PHASE: U[0] = 1; U[3] = 1; cfac = -1.0; break;
        default: rc = -1; cfac = 0; break;
      }
      if (rc) return rc;
      orc_apply(phi, n, g->k, g->locs, U, 0, NULL, NULL);
      for (int64_t i = 0; i < dim; ++i) im[i] = cimag(conj(lam[i]) * phi[i]);
      grad[g->param] += 2.0 * cfac * orc_pairwise_sum(im, dim);
    }
    rc = orc_gate_matrix_dagger(g, th, mats, U);
    if (rc) return rc;
    orc_apply(psi, n, g->k, g->locs, U, g->nctrl, g->ctrl_locs, g->ctrl_vals);
    orc_apply(lam, n, g->k, g->locs, U, g->nctrl, g->ctrl_locs, g->ctrl_vals);
  }
  return rc;
}

int orc_gradient(const cplx* psi0, int n, const orc_gate* gates, int ngates,
                 const double* params, int nparams, const cplx* mats,
                 const orc_term* terms, int nterms, double* grad, double* loss) {
  int64_t dim = (int64_t)1 << n;
  cplx* psi = malloc(sizeof(cplx) * dim);
  cplx* lam = malloc(sizeof(cplx) * dim);
  cplx* phi = malloc(sizeof(cplx) * dim);
  double* im = malloc(sizeof(double) * dim);
  if (!psi || !lam || !phi || !im) { free(psi); free(lam); free(phi); free(im); return -2; }
  int rc = 0;
  memcpy(psi, psi0, sizeof(cplx) * dim);
  for (int p = 0; p < nparams; ++p) grad[p] = 0.0;
  rc = orc_apply_circuit(psi, n, gates, ngates, params, mats, 0);
  if (!rc) rc = orc_expect(psi, n, terms, nterms, loss);
  if (!rc) rc = orc_apply_observable(lam, psi, n, terms, nterms);
  for (int kk = ngates - 1; kk >= 0 && !rc; --kk)
    rc = orc_adjoint_step(psi, lam, phi, im, n, &gates[kk], params, nparams, mats, grad);
  free(psi); free(lam); free(phi); free(im);
  return rc;
}

/* ------------------------------------------------------------------------ */
/* Measurement sampling (Sec. "Instructions on Quantum Registers", measure). */
/* The paper fixes no algorithm; this is the deterministic contract both     */
/* sides implement:                                                          */
/*  p_i = re*re + im*im (separately rounded multiply and add).               */
/*  Level-0 blocks of F = 1024 consecutive p_i, S0[b] = left fold of the     */
/*  block; level-1 blocks of F consecutive S0, S1[c] = left fold; total T =  */
/*  left fold of all S1.  For a uniform u: t = u * T; at each level, walk    */
/*  the values v_j of the chosen parent block starting from the carried      */
/*  prefix acc (0 at the top): acc_{j+1} = acc_j + v_j; choose the first j   */
/*  with acc_j + v_j > t; if none, the last j with v_j > 0 (else the last    */
/*  j); carry acc_j down.  The level-0 choice is the sampled basis index.    */
/* ------------------------------------------------------------------------ */
#define ORC_F 1024

static int64_t walk(const double* v, int64_t len, double t, double* acc) {
  double a = *acc, a_last_pos = *acc;
  int64_t last_pos = -1;
  for (int64_t j = 0; j < len; ++j) {
    double nxt = a + v[j];
    if (nxt > t) { *acc = a; return j; }
    if (v[j] > 0) { last_pos = j; a_last_pos = a; }
    a = nxt;
  }
  if (last_pos >= 0) { *acc = a_last_pos; return last_pos; }
  return len - 1; /* all zero: acc_{len-1} equals the carried prefix */
}

int orc_sample(const cplx* psi, int n, const double* u, int nshots, int64_t* out) {
  int64_t dim = (int64_t)1 << n;
  int64_t nb0 = (dim + ORC_F - 1) / ORC_F;
  int64_t nb1 = (nb0 + ORC_F - 1) / ORC_F;
  double* p = malloc(sizeof(double) * dim);
  double* s0 = malloc(sizeof(double) * nb0);
  double* s1 = malloc(sizeof(double) * nb1);
  if (!p || !s0 || !s1) { free(p); free(s0); free(s1); return -2; }
  for (int64_t i = 0; i < dim; ++i) {
    double re = creal(psi[i]), imv = cimag(psi[i]);
    double r2 = re * re;
    double i2 = imv * imv;
    p[i] = r2 + i2;
  }
  for (int64_t b = 0; b < nb0; ++b) {
    int64_t lo = b * ORC_F, hi = lo + ORC_F < dim ? lo + ORC_F : dim;
    double a = p[lo];
    for (int64_t i = lo + 1; i < hi; ++i) a = a + p[i];
    s0[b] = a;
  }
  for (int64_t c = 0; c < nb1; ++c) {
    int64_t lo = c * ORC_F, hi = lo + ORC_F < nb0 ? lo + ORC_F : nb0;
    double a = s0[lo];
    for (int64_t b = lo + 1; b < hi; ++b) a = a + s0[b];
    s1[c] = a;
  }
  double total = s1[0];
  for (int64_t c = 1; c < nb1; ++c) total = total + s1[c];
  for (int s = 0; s < nshots; ++s) {
    double t = u[s] * total;
    double acc = 0.0;
    int64_t c = walk(s1, nb1, t, &acc);
    int64_t b0 = c * ORC_F, b1 = b0 + ORC_F < nb0 ? b0 + ORC_F : nb0;
    int64_t b = b0 + walk(s0 + b0, b1 - b0, t, &acc);
    int64_t i0 = b * ORC_F, i1 = i0 + ORC_F < dim ? i0 + ORC_F : dim;
    out[s] = i0 + walk(p + i0, i1 - i0, t, &acc);
  }
  free(p); free(s0); free(s1);
  return 0;
}

/* measure! on all qubits: project onto the sampled basis state and renormalise */
void orc_collapse(cplx* psi, int n, int64_t x) {
  int64_t dim = (int64_t)1 << n;
  cplx a = psi[x];
  double r = cabs(a);
  for (int64_t i = 0; i < dim; ++i) psi[i] = 0;
  psi[x] = r > 0 ? a / r : 1.0;
}

/* ------------------------------------------------------------------------ */
/* Seeded measurement (the paper fixes no random source; this is the         */
/* library's contract).  The uniform of draw k (k = 1, 2, ...) is the k-th     */
/* output of SplitMix64 started from `seed` (Steele, Lea and Flood,           */
/* "Fast splittable pseudorandom number generators", OOPSLA 2014, with the    */
/* 64-bit finaliser of Stafford's "Mix13"): the generator's state after k     */
/* steps is seed + k * gamma, gamma = 0x9E3779B97F4A7C15, and the output is    */
/* the finaliser of that state.  u = (x >> 11) * 2^-53 keeps the top 53 bits. */
/* Register r's shot j uses draw k = r * nshots + j + 1.                       */

uint64_t orc_splitmix64(uint64_t seed, uint64_t k) {
  uint64_t z = seed + k * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

void orc_seeded_uniforms(uint64_t seed, uint64_t k0, int64_t count, double* u) {
  for (int64_t i = 0; i < count; ++i)
    u[i] = (double)(orc_splitmix64(seed, k0 + (uint64_t)i + 1) >> 11) * (1.0 / 9007199254740992.0);
}
