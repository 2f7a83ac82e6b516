/*
 * bbc_oracle.c -- plain CPU FP64 oracle for the baryon-baryon four-point
 * correlators of the effective block algorithm (Nemura, arXiv:1510.00903).
 *
 * TEST INFRASTRUCTURE.  Only the tests, the smoke check and the benchmark's
 * CPU-baseline leg load this file; the CUDA library never links it, and it
 * shares no code, header, table or constant with the CUDA library.
 *
 * What it computes (the plain definition, Sec. 2 Eq. 2 and Sec. 3 Eq. for the
 * p-Lambda correlator, generalised to every channel of Sec. 4):
 *
 *   C_{a b a' b'}(r) = sum_X < B1_a(X+r) B2_b(X) Bbar3_a' Bbar4_b' >
 *
 * Each baryon is eps_{c0 c1 c2} (q0 Gamma1 q1) delta q2 with Gamma1 = C gamma5
 * in the Dirac representation (Sec. 2 Eq. for p,n; Sec. 2 Eqs. for Sigma, Xi,
 * Lambda and X_u, X_d, X_s); the source uses the same real tensors (Sec. 3).
 * The decuplet Omega- (Sec. 4 footnote: the same operator form with
 * Gamma1 = C gamma_l, Gamma2 = 1, spatial vector index l) is taken as
 * eta_l eps (s C gamma_l s) s with eta = (i, 1, -i) for l = x, y, z, the
 * phase that makes its tensor real like the octet ones.  The other decuplet
 * baryons take the same form with the flavour-symmetric combinations (a
 * reading: the footnote names only the form): Delta++_l = eta_l eps
 * (u C gamma_l u) u, Sigma*+_l = eta_l [eps (u C gamma_l u) s + 2 eps
 * (u C gamma_l s) u] / sqrt3, Xi*0_l = eta_l [eps (s C gamma_l s) u + 2 eps
 * (s C gamma_l u) s] / sqrt3.
 * The six-quark matrix element is the Wick determinant
 *
 *   < Q1..Q6 Qbar'6..Qbar'1 > = det_{ij} [ delta(f_i, g_j) S_{f_i}(x_i)[xi_i, eta_j] ]
 *
 * (Sec. 3, the expansion printed for p-Lambda is this determinant written
 * out), with Q = (B1 quarks, B2 quarks) in operator order at x = X+r and X,
 * and Q' = (B3 quarks, B4 quarks) at the wall source.
 *
 * How: for every sink baryon b and site x the sink tensor is contracted with
 * three propagators, U_b(x)[a][eta0,eta1,eta2] (a sum over the sink colour
 * and spin indices only -- distributivity, no reordering of the Wick sum).
 * Then, for every (X, r), the flavour-preserving permutations sigma of the
 * determinant (sign sgn sigma) and every non-zero entry of the two source
 * tensors are enumerated explicitly:
 *
 *   C(r) = sum_X sum_sigma sgn(sigma) sum_eta T3(eta0..2) T4(eta3..5)
 *            U_B1(X+r)[eta_sigma(0), eta_sigma(1), eta_sigma(2)]
 *            U_B2(X)  [eta_sigma(3), eta_sigma(4), eta_sigma(5)]
 *
 * This is O(V^2) per channel: no FFT, no baryon blocks, no diagram classes.
 * Identical (eta-pattern) terms are merged by summing their weights, which
 * only regroups equal products.
 *
 * Conventions (readings of the paper where it is silent):
 *  - Dirac representation: gamma4 = diag(1,1,-1,-1), gamma_k = [[0,-i s_k],
 *    [i s_k,0]], gamma5 = gamma1 gamma2 gamma3 gamma4, C = gamma4 gamma2.
 *  - spin/colour packing of a propagator row/column: 3*alpha + c.
 *  - site = x + L*(y + L*z); B1 sits at X + r (periodic).
 *  - only the upper Dirac components (0,1) of the four external spins
 *    (Sec. 5); output spin index s = a + 2*(b + 2*(a' + 2*b')).
 *  - Lambda and Sigma0 keep the quark string (d, s, u) for all X_q terms
 *    (the cyclic reorderings are even, Sec. 2 / Sec. 3 Eq. for p-Lambda).
 *
 * Parity status: pinned by the tests (brute-force 6x6 determinants, closed
 * form for plane-wave propagators, SU(3) and spin-rotation invariance,
 * Grassmann antisymmetry, isospin zeros, homogeneity).
 */
#include <complex.h>
#include <math.h>
#include <omp.h>
#include <stdlib.h>
#include <string.h>

typedef double _Complex cplx;

enum { FL_U = 0, FL_D = 1, FL_S = 2 };

/* One baryon operator: quark string flavours, its diquark matrix Gamma1
 * (gam: 0 = C gamma5, 1..3 = eta_l C gamma_l) and up to three terms
 * coef * eps(c0,c1,c2) * Gamma1(a_i, a_j) * delta(ext, a_k). */
typedef struct {
  const char* name;
  int flav[3];
  int gam;
  int nterm;
  double coef[3];
  int gi[3], gj[3], dk[3];
} baryon_t;

enum { B_P, B_N, B_SP, B_SM, B_S0, B_L, B_X0, B_XM, B_OX, B_OY, B_OZ, B_DX, B_DY, B_DZ, B_SSX, B_SSY, B_SSZ,
       B_XSX, B_XSY, B_XSZ, NBARYON };

static baryon_t g_bar[NBARYON];

/* channel = sink (B1, B2), source (B3, B4); 52 printed channels (Sec. 4,
 * Eqs. GeneralBB_NN ... GeneralBB_XX), the four channels the paper omits
 * because they vanish in the isospin limit, then eight other charge states
 * (pp, nn, S+S+, S-S-, X0X0, X-X-, pS+, nS-, each onto itself), then the
 * decuplet channels of the Sec. 4 footnote: Omega_l1 Omega_l2 <- Omega_l3
 * Omega_l4 at id 64 + 27 l1 + 9 l2 + 3 l3 + l4 and p Omega_l <- p Omega_l'
 * at id 145 + 3 l + l' (l = 0, 1, 2 for x, y, z); the same 81 vector
 * combinations of Delta++ Delta++ at 154 + ..., Sigma*+ Sigma*+ at 235 + ...
 * and Xi*0 Xi*0 at 316 + ..., and p Delta++_l <- p Delta++_l' at
 * 397 + 3 l + l'. */
typedef struct { int b[4]; const char* name; } channel_t;
#define NCHAN_ALL 406
static channel_t g_chan[NCHAN_ALL];
static int g_nchan = 0;

static double g_gam[4][4][4]; /* [0] = C gamma5, [l] = eta_l C gamma_l */
static int g_gam_ok = 1;      /* every eta_l C gamma_l came out real */
static int g_init = 0;

static void add_chan(int b1, int b2, int b3, int b4) {
  g_chan[g_nchan].b[0] = b1; g_chan[g_nchan].b[1] = b2;
  g_chan[g_nchan].b[2] = b3; g_chan[g_nchan].b[3] = b4;
  g_nchan++;
}

static void set_bar(int id, const char* name, int f0, int f1, int f2) {
  g_bar[id].name = name;
  g_bar[id].flav[0] = f0; g_bar[id].flav[1] = f1; g_bar[id].flav[2] = f2;
  g_bar[id].gam = 0;
  g_bar[id].nterm = 0;
}
static void add_term(int id, double coef, int gi, int gj, int dk) {
  baryon_t* b = &g_bar[id];
  b->coef[b->nterm] = coef; b->gi[b->nterm] = gi; b->gj[b->nterm] = gj; b->dk[b->nterm] = dk;
  b->nterm++;
}

static void matmul4(cplx a[4][4], cplx b[4][4], cplx c[4][4]) {
  for (int i = 0; i < 4; i++)
    for (int j = 0; j < 4; j++) {
      cplx s = 0;
      for (int k = 0; k < 4; k++) s += a[i][k] * b[k][j];
      c[i][j] = s;
    }
}

static void init_tables(void) {
  if (g_init) return;
  /* Dirac matrices and C gamma5 from their definitions. */
  cplx g[5][4][4];
  memset(g, 0, sizeof(g));
  /* Pauli matrices */
  cplx s[3][2][2] = {{{0, 1}, {1, 0}}, {{0, -I}, {I, 0}}, {{1, 0}, {0, -1}}};
  for (int k = 0; k < 3; k++)
    for (int i = 0; i < 2; i++)
      for (int j = 0; j < 2; j++) {
        g[k][i][2 + j] = -I * s[k][i][j];
        g[k][2 + i][j] = I * s[k][i][j];
      }
  g[3][0][0] = 1; g[3][1][1] = 1; g[3][2][2] = -1; g[3][3][3] = -1;
  cplx t1[4][4], t2[4][4], g5[4][4], cm[4][4], cg5[4][4];
  matmul4(g[0], g[1], t1);
  matmul4(t1, g[2], t2);
  matmul4(t2, g[3], g5);
  matmul4(g[3], g[1], cm); /* C = gamma4 gamma2 */
  matmul4(cm, g5, cg5);
  for (int i = 0; i < 4; i++)
    for (int j = 0; j < 4; j++) g_gam[0][i][j] = creal(cg5[i][j]);
  /* eta_l C gamma_l, eta = (i, 1, -i): real symmetric matrices */
  const cplx eta[3] = {I, 1, -I};
  for (int l = 0; l < 3; l++) {
    cplx cgl[4][4];
    matmul4(cm, g[l], cgl);
    for (int i = 0; i < 4; i++)
      for (int j = 0; j < 4; j++) {
        const cplx v = eta[l] * cgl[i][j];
        if (cimag(v) != 0.0) g_gam_ok = 0;
        g_gam[1 + l][i][j] = creal(v);
      }
  }

  const double r6 = 1.0 / sqrt(6.0), r2 = 1.0 / sqrt(2.0);
  set_bar(B_P, "p", FL_U, FL_D, FL_U);    add_term(B_P, +1.0, 0, 1, 2);
  set_bar(B_N, "n", FL_U, FL_D, FL_D);    add_term(B_N, -1.0, 0, 1, 2);
  set_bar(B_SP, "Sigma+", FL_U, FL_S, FL_U); add_term(B_SP, -1.0, 0, 1, 2);
  set_bar(B_SM, "Sigma-", FL_D, FL_S, FL_D); add_term(B_SM, -1.0, 0, 1, 2);
  set_bar(B_X0, "Xi0", FL_U, FL_S, FL_S); add_term(B_X0, +1.0, 0, 1, 2);
  set_bar(B_XM, "Xi-", FL_D, FL_S, FL_S); add_term(B_XM, -1.0, 0, 1, 2);
  /* Lambda = (X_u + X_d - 2 X_s)/sqrt6, Sigma0 = (X_u - X_d)/sqrt2, string (d,s,u):
   * X_u = eps (d Cg5 s) u, X_d = eps (s Cg5 u) d, X_s = eps (u Cg5 d) s. */
  set_bar(B_L, "Lambda", FL_D, FL_S, FL_U);
  add_term(B_L, r6, 0, 1, 2); add_term(B_L, r6, 1, 2, 0); add_term(B_L, -2.0 * r6, 2, 0, 1);
  set_bar(B_S0, "Sigma0", FL_D, FL_S, FL_U);
  add_term(B_S0, r2, 0, 1, 2); add_term(B_S0, -r2, 1, 2, 0);
  /* Omega-_l = eta_l eps (s C gamma_l s) s (Sec. 4 footnote) */
  {
    const int ids[3] = {B_OX, B_OY, B_OZ};
    const char* names[3] = {"Omega_x", "Omega_y", "Omega_z"};
    for (int l = 0; l < 3; l++) {
      set_bar(ids[l], names[l], FL_S, FL_S, FL_S);
      g_bar[ids[l]].gam = 1 + l;
      add_term(ids[l], 1.0, 0, 1, 2);
    }
  }
  /* Delta++_l = eta_l eps (u C gamma_l u) u; Sigma*+_l on the string (u, u, s):
   * [eps (q0 G q1) q2 + 2 eps (q0 G q2) q1] / sqrt3; Xi*0_l the same on (s, s, u) */
  {
    const double r3 = 1.0 / sqrt(3.0);
    const char* dn[3] = {"Delta++_x", "Delta++_y", "Delta++_z"};
    const char* sn[3] = {"Sigma*+_x", "Sigma*+_y", "Sigma*+_z"};
    const char* xn[3] = {"Xi*0_x", "Xi*0_y", "Xi*0_z"};
    for (int l = 0; l < 3; l++) {
      set_bar(B_DX + l, dn[l], FL_U, FL_U, FL_U);
      g_bar[B_DX + l].gam = 1 + l;
      add_term(B_DX + l, 1.0, 0, 1, 2);
      set_bar(B_SSX + l, sn[l], FL_U, FL_U, FL_S);
      g_bar[B_SSX + l].gam = 1 + l;
      add_term(B_SSX + l, r3, 0, 1, 2);
      add_term(B_SSX + l, 2.0 * r3, 0, 2, 1);
      set_bar(B_XSX + l, xn[l], FL_S, FL_S, FL_U);
      g_bar[B_XSX + l].gam = 1 + l;
      add_term(B_XSX + l, r3, 0, 1, 2);
      add_term(B_XSX + l, 2.0 * r3, 0, 2, 1);
    }
  }

  /* 52 channels in printed order */
  g_nchan = 0;
  add_chan(B_P, B_N, B_P, B_N);
  {
    int nl[3][2] = {{B_P, B_L}, {B_SP, B_N}, {B_S0, B_P}};
    for (int a = 0; a < 3; a++)
      for (int b = 0; b < 3; b++) add_chan(nl[a][0], nl[a][1], nl[b][0], nl[b][1]);
  }
  {
    int src6[6][2] = {{B_L, B_L}, {B_P, B_XM}, {B_N, B_X0}, {B_SP, B_SM}, {B_S0, B_S0}, {B_S0, B_L}};
    for (int b = 0; b < 5; b++) add_chan(B_L, B_L, src6[b][0], src6[b][1]);
    for (int b = 0; b < 6; b++) add_chan(B_P, B_XM, src6[b][0], src6[b][1]);
    for (int b = 0; b < 6; b++) add_chan(B_N, B_X0, src6[b][0], src6[b][1]);
    for (int b = 0; b < 6; b++) add_chan(B_SP, B_SM, src6[b][0], src6[b][1]);
    for (int b = 0; b < 5; b++) add_chan(B_S0, B_S0, src6[b][0], src6[b][1]);
    for (int b = 1; b < 4; b++) add_chan(B_S0, B_L, src6[b][0], src6[b][1]);
    add_chan(B_S0, B_L, B_S0, B_L);
  }
  {
    int xl[3][2] = {{B_XM, B_L}, {B_SM, B_X0}, {B_S0, B_XM}};
    for (int a = 0; a < 3; a++)
      for (int b = 0; b < 3; b++) add_chan(xl[a][0], xl[a][1], xl[b][0], xl[b][1]);
  }
  add_chan(B_XM, B_X0, B_XM, B_X0);
  /* the four omitted channels (zero in the isospin limit) */
  add_chan(B_L, B_L, B_S0, B_L);
  add_chan(B_S0, B_S0, B_S0, B_L);
  add_chan(B_S0, B_L, B_L, B_L);
  add_chan(B_S0, B_L, B_S0, B_S0);
  /* other charge states (Sec. 4 footnote), ids 56..63 */
  add_chan(B_P, B_P, B_P, B_P);
  add_chan(B_N, B_N, B_N, B_N);
  add_chan(B_SP, B_SP, B_SP, B_SP);
  add_chan(B_SM, B_SM, B_SM, B_SM);
  add_chan(B_X0, B_X0, B_X0, B_X0);
  add_chan(B_XM, B_XM, B_XM, B_XM);
  add_chan(B_P, B_SP, B_P, B_SP);
  add_chan(B_N, B_SM, B_N, B_SM);
  /* decuplet channels (Sec. 4 footnote), ids 64..153 */
  {
    const int om[3] = {B_OX, B_OY, B_OZ};
    for (int l1 = 0; l1 < 3; l1++)
      for (int l2 = 0; l2 < 3; l2++)
        for (int l3 = 0; l3 < 3; l3++)
          for (int l4 = 0; l4 < 3; l4++) add_chan(om[l1], om[l2], om[l3], om[l4]);
    for (int l = 0; l < 3; l++)
      for (int m = 0; m < 3; m++) add_chan(B_P, om[l], B_P, om[m]);
  }
  /* ids 154..405: Delta++, Sigma*+, Xi*0 pairs (81 vector combinations each), p Delta++ */
  {
    const int base[3] = {B_DX, B_SSX, B_XSX};
    for (int f = 0; f < 3; f++)
      for (int l1 = 0; l1 < 3; l1++)
        for (int l2 = 0; l2 < 3; l2++)
          for (int l3 = 0; l3 < 3; l3++)
            for (int l4 = 0; l4 < 3; l4++) add_chan(base[f] + l1, base[f] + l2, base[f] + l3, base[f] + l4);
    for (int l = 0; l < 3; l++)
      for (int m = 0; m < 3; m++) add_chan(B_P, B_DX + l, B_P, B_DX + m);
  }
  g_init = 1;
}

/* ---- public helpers ---------------------------------------------------- */

int oracle_channel_count(void) { init_tables(); return g_nchan; }

/* OpenMP threads the parallel loops over X use (the timing reports it). */
int oracle_threads(void) { return omp_get_max_threads(); }

int oracle_channel_baryons(int ch, int* out4) {
  init_tables();
  if (ch < 0 || ch >= g_nchan) return -1;
  for (int i = 0; i < 4; i++) out4[i] = g_chan[ch].b[i];
  return 0;
}

const char* oracle_baryon_name(int b) {
  init_tables();
  return (b >= 0 && b < NBARYON) ? g_bar[b].name : "";
}

void oracle_cg5(double* out16) {
  init_tables();
  for (int i = 0; i < 4; i++)
    for (int j = 0; j < 4; j++) out16[4 * i + j] = g_gam[0][i][j];
}

/* Diquark matrix gam (0 = C gamma5, 1..3 = eta_l C gamma_l) as used by the
 * tensors; returns -1 for a bad index or if eta_l C gamma_l was not real. */
int oracle_gamma(int gam, double* out16) {
  init_tables();
  if (gam < 0 || gam > 3 || !g_gam_ok) return -1;
  for (int i = 0; i < 4; i++)
    for (int j = 0; j < 4; j++) out16[4 * i + j] = g_gam[gam][i][j];
  return 0;
}

/* Dense baryon tensor T_b(ext; q0, q1, q2) over 12^3 (index 144*q0 + 12*q1 + q2,
 * q = 3*spin + colour), Dirac index ext in {0..3}.  Shared by sink and source. */
static void baryon_tensor(int b, int ext, double* T /* 1728 */) {
  static const int eps_p[6][3] = {{0, 1, 2}, {1, 2, 0}, {2, 0, 1}, {0, 2, 1}, {2, 1, 0}, {1, 0, 2}};
  static const double eps_s[6] = {1, 1, 1, -1, -1, -1};
  memset(T, 0, sizeof(double) * 1728);
  const baryon_t* B = &g_bar[b];
  for (int t = 0; t < B->nterm; t++)
    for (int e = 0; e < 6; e++)
      for (int ai = 0; ai < 4; ai++)
        for (int aj = 0; aj < 4; aj++) {
          double g = g_gam[B->gam][ai][aj];
          if (g == 0.0) continue;
          int sp[3];
          sp[B->gi[t]] = ai; sp[B->gj[t]] = aj; sp[B->dk[t]] = ext;
          int q0 = 3 * sp[0] + eps_p[e][0], q1 = 3 * sp[1] + eps_p[e][1], q2 = 3 * sp[2] + eps_p[e][2];
          T[144 * q0 + 12 * q1 + q2] += B->coef[t] * eps_s[e] * g;
        }
}

/* U_b(x)[a][eta] for all sites: out[(x*2 + a)*1728 + eta], sink spin
 * a + off (off = 0: upper components, 2: lower components). */
static void sink_tensor_field(int b, int V, const cplx* const S[3], int off, cplx* U) {
  double T[2][1728];
  baryon_tensor(b, off, T[0]);
  baryon_tensor(b, off + 1, T[1]);
  const int* fl = g_bar[b].flav;
#pragma omp parallel for schedule(static)
  for (int x = 0; x < V; x++) {
    const cplx* s0 = S[fl[0]] + (size_t)x * 144;
    const cplx* s1 = S[fl[1]] + (size_t)x * 144;
    const cplx* s2 = S[fl[2]] + (size_t)x * 144;
    for (int a = 0; a < 2; a++) {
      cplx* u = U + ((size_t)x * 2 + a) * 1728;
      for (int i = 0; i < 1728; i++) u[i] = 0;
      for (int xi = 0; xi < 1728; xi++) {
        double w = T[a][xi];
        if (w == 0.0) continue;
        int r0 = xi / 144, r1 = (xi / 12) % 12, r2 = xi % 12;
        for (int e0 = 0; e0 < 12; e0++) {
          cplx p0 = w * s0[12 * r0 + e0];
          for (int e1 = 0; e1 < 12; e1++) {
            cplx p01 = p0 * s1[12 * r1 + e1];
            cplx* ue = u + 144 * e0 + 12 * e1;
            for (int e2 = 0; e2 < 12; e2++) ue[e2] += p01 * s2[12 * r2 + e2];
          }
        }
      }
    }
  }
}

typedef struct { int i1, i2; double w; } term_t;

static int cmp_term(const void* a, const void* b) {
  const term_t* x = (const term_t*)a;
  const term_t* y = (const term_t*)b;
  if (x->i1 != y->i1) return x->i1 < y->i1 ? -1 : 1;
  if (x->i2 != y->i2) return x->i2 < y->i2 ? -1 : 1;
  return 0;
}

/* Flavour-preserving permutations of the Wick determinant.  perm[k][i] = source
 * position contracted with sink position i; sign = parity. */
static int wick_perms(const int sinkf[6], const int srcf[6], int perm[720][6], int sign[720]) {
  int p[6] = {0, 1, 2, 3, 4, 5}, n = 0;
  /* Heap-free enumeration: iterate over all 6! index tuples in lexicographic order. */
  for (int a0 = 0; a0 < 6; a0++)
    for (int a1 = 0; a1 < 6; a1++)
      for (int a2 = 0; a2 < 6; a2++)
        for (int a3 = 0; a3 < 6; a3++)
          for (int a4 = 0; a4 < 6; a4++)
            for (int a5 = 0; a5 < 6; a5++) {
              int q[6] = {a0, a1, a2, a3, a4, a5}, used = 0, ok = 1;
              for (int i = 0; i < 6; i++) {
                if (used & (1 << q[i])) { ok = 0; break; }
                used |= 1 << q[i];
                if (sinkf[i] != srcf[q[i]]) { ok = 0; break; }
              }
              if (!ok) continue;
              int inv = 0;
              for (int i = 0; i < 6; i++)
                for (int j = i + 1; j < 6; j++) inv += q[i] > q[j];
              for (int i = 0; i < 6; i++) perm[n][i] = q[i];
              sign[n] = (inv & 1) ? -1 : 1;
              n++;
            }
  (void)p;
  return n;
}

/* Number of flavour-preserving Wick permutations of a channel (pin helper). */
int oracle_wick_count(int ch) {
  init_tables();
  if (ch < 0 || ch >= g_nchan) return -1;
  int sf[6], gf[6];
  for (int i = 0; i < 3; i++) {
    sf[i] = g_bar[g_chan[ch].b[0]].flav[i]; sf[3 + i] = g_bar[g_chan[ch].b[1]].flav[i];
    gf[i] = g_bar[g_chan[ch].b[2]].flav[i]; gf[3 + i] = g_bar[g_chan[ch].b[3]].flav[i];
  }
  static int perm[720][6], sign[720];
  return wick_perms(sf, gf, perm, sign);
}

/* Term list of one channel and one pair of source spins (a', b') (Dirac
 * indices). */
static term_t* build_terms(int ch, int ap, int bp, int* nout) {
  const channel_t* C = &g_chan[ch];
  int sf[6], gf[6];
  for (int i = 0; i < 3; i++) {
    sf[i] = g_bar[C->b[0]].flav[i]; sf[3 + i] = g_bar[C->b[1]].flav[i];
    gf[i] = g_bar[C->b[2]].flav[i]; gf[3 + i] = g_bar[C->b[3]].flav[i];
  }
  int perm[720][6], sign[720];
  int np = wick_perms(sf, gf, perm, sign);
  double T3[1728], T4[1728];
  baryon_tensor(C->b[2], ap, T3);
  baryon_tensor(C->b[3], bp, T4);
  int nz3 = 0, nz4 = 0, z3[1728], z4[1728];
  for (int i = 0; i < 1728; i++) {
    if (T3[i] != 0.0) z3[nz3++] = i;
    if (T4[i] != 0.0) z4[nz4++] = i;
  }
  size_t cap = (size_t)np * nz3 * nz4;
  term_t* t = (term_t*)malloc(sizeof(term_t) * (cap ? cap : 1));
  size_t n = 0;
  for (int k = 0; k < np; k++)
    for (int i3 = 0; i3 < nz3; i3++)
      for (int i4 = 0; i4 < nz4; i4++) {
        int e[6];
        e[0] = z3[i3] / 144; e[1] = (z3[i3] / 12) % 12; e[2] = z3[i3] % 12;
        e[3] = z4[i4] / 144; e[4] = (z4[i4] / 12) % 12; e[5] = z4[i4] % 12;
        const int* s = perm[k];
        t[n].i1 = 144 * e[s[0]] + 12 * e[s[1]] + e[s[2]];
        t[n].i2 = 144 * e[s[3]] + 12 * e[s[4]] + e[s[5]];
        t[n].w = sign[k] * T3[z3[i3]] * T4[z4[i4]];
        n++;
      }
  /* merge equal (i1, i2) terms */
  qsort(t, n, sizeof(term_t), cmp_term);
  size_t m = 0;
  for (size_t i = 0; i < n; i++) {
    if (m > 0 && t[m - 1].i1 == t[i].i1 && t[m - 1].i2 == t[i].i2) t[m - 1].w += t[i].w;
    else t[m++] = t[i];
  }
  size_t w = 0;
  for (size_t i = 0; i < m; i++)
    if (t[i].w != 0.0) t[w++] = t[i];
  *nout = (int)w;
  return t;
}

static int correlator_impl(int L, const cplx* Su, const cplx* Sd, const cplx* Ss, int n_ch, const int* channels,
                           int n_r, const int* r_list, int lower, cplx* out);

/*
 * oracle_correlator: one time slice, raw (un-normalised) correlators of the
 * upper Dirac components.
 *   L: spatial extent (V = L^3 sites)
 *   Su, Sd, Ss: propagators [V][12][12] complex128 (Su may equal Sd)
 *   channels[n_ch]: channel ids (0..51 printed order, 52..55 omitted channels,
 *     56..63 other charge states, 64..144 Omega Omega, 145..153 p Omega,
 *     154..234 Delta++ Delta++, 235..315 Sigma*+ Sigma*+, 316..396 Xi*0 Xi*0,
 *     397..405 p Delta++)
 *   r_list[n_r]: output sites r (site index), or n_r <= 0 for all V sites
 *   out: [n_ch][n_r or V][16] complex128, spin s = a + 2(b + 2(a' + 2 b'))
 * Returns 0, or -1 on a bad argument, -2 on allocation failure.
 */
int oracle_correlator(int L, const cplx* Su, const cplx* Sd, const cplx* Ss, int n_ch,
                      const int* channels, int n_r, const int* r_list, cplx* out) {
  return correlator_impl(L, Su, Sd, Ss, n_ch, channels, n_r, r_list, 0, out);
}

/*
 * oracle_correlator_components: as oracle_correlator, for the upper
 * (lower = 0: Dirac indices 0, 1) or the lower (lower = 1: Dirac indices
 * 2, 3) two components of all four external spinor indices (Sec. 5: upper
 * components give the positive-parity baryons forward in time, lower ones
 * the antibaryons backward in time).  Output spins relabelled to 0, 1:
 * s = a~ + 2(b~ + 2(a~' + 2 b~')) with a = a~ + 2 lower.
 */
int oracle_correlator_components(int L, const cplx* Su, const cplx* Sd, const cplx* Ss, int n_ch,
                                 const int* channels, int n_r, const int* r_list, int lower, cplx* out) {
  if (lower != 0 && lower != 1) return -1;
  return correlator_impl(L, Su, Sd, Ss, n_ch, channels, n_r, r_list, lower, out);
}

static int correlator_impl(int L, const cplx* Su, const cplx* Sd, const cplx* Ss, int n_ch, const int* channels,
                           int n_r, const int* r_list, int lower, cplx* out) {
  init_tables();
  const int off = 2 * lower;
  if (L < 1 || n_ch < 0 || !g_gam_ok) return -1;
  for (int c = 0; c < n_ch; c++)
    if (channels[c] < 0 || channels[c] >= g_nchan) return -1;
  const int V = L * L * L;
  int all_r = n_r <= 0;
  int nr = all_r ? V : n_r;
  int* rl = (int*)malloc(sizeof(int) * nr);
  if (!rl) return -2;
  for (int i = 0; i < nr; i++) {
    rl[i] = all_r ? i : r_list[i];
    if (rl[i] < 0 || rl[i] >= V) { free(rl); return -1; }
  }
  const cplx* S[3] = {Su, Sd, Ss};
  /* sink tensor fields of every sink baryon used */
  cplx* U[NBARYON] = {0};
  for (int c = 0; c < n_ch; c++)
    for (int k = 0; k < 2; k++) {
      int b = g_chan[channels[c]].b[k];
      if (!U[b]) {
        U[b] = (cplx*)malloc(sizeof(cplx) * (size_t)V * 2 * 1728);
        if (!U[b]) { free(rl); return -2; }
        sink_tensor_field(b, V, S, off, U[b]);
      }
    }
  memset(out, 0, sizeof(cplx) * (size_t)n_ch * nr * 16);
  for (int c = 0; c < n_ch; c++) {
    const channel_t* C = &g_chan[channels[c]];
    const cplx* U1 = U[C->b[0]];
    const cplx* U2 = U[C->b[1]];
    int nt[4];
    term_t* tl[4];
    for (int sp = 0; sp < 4; sp++) tl[sp] = build_terms(channels[c], off + (sp & 1), off + (sp >> 1), &nt[sp]);
    cplx* o = out + (size_t)c * nr * 16;
#pragma omp parallel for schedule(dynamic, 1)
    for (int ir = 0; ir < nr; ir++) {
      int r = rl[ir], rx = r % L, ry = (r / L) % L, rz = r / (L * L);
      cplx acc[16];
      for (int s = 0; s < 16; s++) acc[s] = 0;
      for (int X = 0; X < V; X++) {
        int x = X % L, y = (X / L) % L, z = X / (L * L);
        int Xr = (x + rx) % L + L * ((y + ry) % L + L * ((z + rz) % L));
        const cplx* u1a = U1 + (size_t)Xr * 2 * 1728;
        const cplx* u2a = U2 + (size_t)X * 2 * 1728;
        for (int sp = 0; sp < 4; sp++) {
          cplx a00 = 0, a01 = 0, a10 = 0, a11 = 0; /* (a, b) */
          const term_t* t = tl[sp];
          for (int k = 0; k < nt[sp]; k++) {
            cplx p0 = t[k].w * u1a[t[k].i1], p1 = t[k].w * u1a[1728 + t[k].i1];
            cplx q0 = u2a[t[k].i2], q1 = u2a[1728 + t[k].i2];
            a00 += p0 * q0; a10 += p1 * q0; a01 += p0 * q1; a11 += p1 * q1;
          }
          /* s = a + 2 b + 4 a' + 8 b' ; sp = a' + 2 b' */
          acc[0 + 4 * sp] += a00; acc[1 + 4 * sp] += a10;
          acc[2 + 4 * sp] += a01; acc[3 + 4 * sp] += a11;
        }
      }
      for (int s = 0; s < 16; s++) o[(size_t)ir * 16 + s] = acc[s];
    }
    for (int sp = 0; sp < 4; sp++) free(tl[sp]);
  }
  for (int b = 0; b < NBARYON; b++) free(U[b]);
  free(rl);
  return 0;
}

/* Number of merged (i1, i2) terms for a channel and source spin pair. */
int oracle_term_count(int ch, int ap, int bp) {
  init_tables();
  if (ch < 0 || ch >= g_nchan) return -1;
  int n;
  term_t* t = build_terms(ch, ap, bp, &n);
  free(t);
  return n;
}
