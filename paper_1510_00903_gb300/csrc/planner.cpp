// planner.cpp -- diagram classification, block aggregation and contraction
// plan of the effective block algorithm (arXiv:1510.00903, Secs. 3-4 and
// Appendix A).  Host C++, no CUDA.
//
// Per channel <B1 B2 | Bbar3 Bbar4> and per pair of source operator terms
// (the X_u, X_d, X_s terms of Lambda and Sigma0 are taken one at a time, as in
// the paper's Tables), the flavour-preserving Wick permutations are grouped
// into diagrams by the set S1 of source quarks contracted into the sink baryon
// B1 (identical quarks of one sink baryon are absorbed into its block, Sec. 3
// factor 2^{B - N_Lambda - N_Sigma0}).  A source baryon whose quarks split 2+1
// between the sink baryons puts its tensor into the block holding two of them;
// the third (minority) quark becomes an open index of both blocks: colour only
// when it is the quark carried by delta (its spin is then the external source
// spin, which moves to the other block), colour and spin otherwise (Sec. 3,
// diagrams (ii)-(vi)).  Each block is a sparse integer-weighted sum over the
// entries of four per-site sink tensor families; identical blocks (up to the
// order of their external and open axes and an overall sign) are stored once
// (Appendix A), and so are identical aligned block-pair products.
#include "planner.hpp"

#include <algorithm>
#include <array>
#include <cmath>
#include <map>
#include <numeric>
#include <tuple>
#include <utility>

namespace bbc {
namespace {

struct Term {
  int coef, gi, gj, dk;  // coef * eps * Gamma1(a_gi, a_gj) * delta(ext, a_dk)
  int g;                 // Gamma1: 0 = C gamma5, 1..3 = eta_l C gamma_l (l = x, y, z)
};
struct Op {
  const char* name;
  char flav[4];  // quark string (u, d, s)
  double scale;  // operator prefactor (sign, 1/sqrt6, 1/sqrt2)
  int nterm;
  Term t[3];
  int n_s;  // strange quarks
};

// Sec. 2: p, n (Eq. FieldOperator_N); Sigma+-, Sigma0, Lambda, Xi0, Xi-
// (Eq. FieldOperator_SLXi) with X_u = eps(d Cg5 s)u, X_d = eps(s Cg5 u)d,
// X_s = eps(u Cg5 d)s (Eq. FieldOperator_xxx) written on the common string
// (d, s, u) (cyclic reorderings of three quark fields are even).
// The decuplet Omega-_l of the Sec. 4 footnote (the same operator form with
// Gamma1 = C gamma_l, Gamma2 = 1) is eta_l eps (s C gamma_l s) s with
// eta = (i, 1, -i), the phase that makes its matrix real.  The other
// decuplet baryons take the same form with the flavour-symmetric
// combinations: Delta++_l = eta_l eps (u C gamma_l u) u, Sigma*+_l =
// eta_l [eps (u C gamma_l u) s + 2 eps (u C gamma_l s) u] / sqrt3 and Xi*0_l
// = eta_l [eps (s C gamma_l s) u + 2 eps (s C gamma_l u) s] / sqrt3, the
// latter two on the strings (u, u, s) and (s, s, u).
enum { OP_P, OP_N, OP_SP, OP_SM, OP_S0, OP_LA, OP_X0, OP_XM, OP_OX, OP_OY, OP_OZ, OP_DX = 11, OP_SSX = 14,
       OP_XSX = 17, N_OP = 20 };
const double kInvSqrt6 = 0.40824829046386301637;
const double kInvSqrt2 = 0.70710678118654752440;
const double kInvSqrt3 = 0.57735026918962576451;
const Op kOps[N_OP] = {
    {"p", "udu", 1.0, 1, {{1, 0, 1, 2}}, 0},
    {"n", "udd", -1.0, 1, {{1, 0, 1, 2}}, 0},
    {"Sigma+", "usu", -1.0, 1, {{1, 0, 1, 2}}, 1},
    {"Sigma-", "dsd", -1.0, 1, {{1, 0, 1, 2}}, 1},
    {"Sigma0", "dsu", kInvSqrt2, 2, {{1, 0, 1, 2}, {-1, 1, 2, 0}}, 1},
    {"Lambda", "dsu", kInvSqrt6, 3, {{1, 0, 1, 2}, {1, 1, 2, 0}, {-2, 2, 0, 1}}, 1},
    {"Xi0", "uss", 1.0, 1, {{1, 0, 1, 2}}, 2},
    {"Xi-", "dss", -1.0, 1, {{1, 0, 1, 2}}, 2},
    {"Omega_x", "sss", 1.0, 1, {{1, 0, 1, 2, 1}}, 3},
    {"Omega_y", "sss", 1.0, 1, {{1, 0, 1, 2, 2}}, 3},
    {"Omega_z", "sss", 1.0, 1, {{1, 0, 1, 2, 3}}, 3},
    {"Delta++_x", "uuu", 1.0, 1, {{1, 0, 1, 2, 1}}, 0},
    {"Delta++_y", "uuu", 1.0, 1, {{1, 0, 1, 2, 2}}, 0},
    {"Delta++_z", "uuu", 1.0, 1, {{1, 0, 1, 2, 3}}, 0},
    {"Sigma*+_x", "uus", kInvSqrt3, 2, {{1, 0, 1, 2, 1}, {2, 0, 2, 1, 1}}, 1},
    {"Sigma*+_y", "uus", kInvSqrt3, 2, {{1, 0, 1, 2, 2}, {2, 0, 2, 1, 2}}, 1},
    {"Sigma*+_z", "uus", kInvSqrt3, 2, {{1, 0, 1, 2, 3}, {2, 0, 2, 1, 3}}, 1},
    {"Xi*0_x", "ssu", kInvSqrt3, 2, {{1, 0, 1, 2, 1}, {2, 0, 2, 1, 1}}, 2},
    {"Xi*0_y", "ssu", kInvSqrt3, 2, {{1, 0, 1, 2, 2}, {2, 0, 2, 1, 2}}, 2},
    {"Xi*0_z", "ssu", kInvSqrt3, 2, {{1, 0, 1, 2, 3}, {2, 0, 2, 1, 3}}, 2},
};

// Channels of Sec. 4 (Eqs. GeneralBB_NN .. GeneralBB_XX) in printed order,
// then the four omitted ones, eight other charge states, and the decuplet
// channels: Omega_l1 Omega_l2 <- Omega_l3 Omega_l4 at 64 + 27 l1 + 9 l2 +
// 3 l3 + l4, p Omega_l <- p Omega_l' at 145 + 3 l + l'; the same 81 vector
// combinations for Delta++ Delta++ (154 + ...), Sigma*+ Sigma*+ (235 + ...)
// and Xi*0 Xi*0 (316 + ...), then p Delta++_l <- p Delta++_l' at 397 + 3 l + l'.
std::vector<std::array<int, 4>> make_channels() {
  std::vector<std::array<int, 4>> c;
  c.push_back({OP_P, OP_N, OP_P, OP_N});
  const int nl[3][2] = {{OP_P, OP_LA}, {OP_SP, OP_N}, {OP_S0, OP_P}};
  for (auto& a : nl)
    for (auto& b : nl) c.push_back({a[0], a[1], b[0], b[1]});
  const int s6[6][2] = {{OP_LA, OP_LA}, {OP_P, OP_XM}, {OP_N, OP_X0},
                        {OP_SP, OP_SM}, {OP_S0, OP_S0}, {OP_S0, OP_LA}};
  for (int b = 0; b < 5; b++) c.push_back({OP_LA, OP_LA, s6[b][0], s6[b][1]});
  const int mid[3][2] = {{OP_P, OP_XM}, {OP_N, OP_X0}, {OP_SP, OP_SM}};
  for (auto& a : mid)
    for (int b = 0; b < 6; b++) c.push_back({a[0], a[1], s6[b][0], s6[b][1]});
  for (int b = 0; b < 5; b++) c.push_back({OP_S0, OP_S0, s6[b][0], s6[b][1]});
  for (int b = 1; b < 4; b++) c.push_back({OP_S0, OP_LA, s6[b][0], s6[b][1]});
  c.push_back({OP_S0, OP_LA, OP_S0, OP_LA});
  const int xl[3][2] = {{OP_XM, OP_LA}, {OP_SM, OP_X0}, {OP_S0, OP_XM}};
  for (auto& a : xl)
    for (auto& b : xl) c.push_back({a[0], a[1], b[0], b[1]});
  c.push_back({OP_XM, OP_X0, OP_XM, OP_X0});
  c.push_back({OP_LA, OP_LA, OP_S0, OP_LA});
  c.push_back({OP_S0, OP_S0, OP_S0, OP_LA});
  c.push_back({OP_S0, OP_LA, OP_LA, OP_LA});
  c.push_back({OP_S0, OP_LA, OP_S0, OP_S0});
  // other charge states (Sec. 4 footnote: the extension is the same
  // construction with other operators): ids 56..63
  c.push_back({OP_P, OP_P, OP_P, OP_P});
  c.push_back({OP_N, OP_N, OP_N, OP_N});
  c.push_back({OP_SP, OP_SP, OP_SP, OP_SP});
  c.push_back({OP_SM, OP_SM, OP_SM, OP_SM});
  c.push_back({OP_X0, OP_X0, OP_X0, OP_X0});
  c.push_back({OP_XM, OP_XM, OP_XM, OP_XM});
  c.push_back({OP_P, OP_SP, OP_P, OP_SP});
  c.push_back({OP_N, OP_SM, OP_N, OP_SM});
  const int om[3] = {OP_OX, OP_OY, OP_OZ};
  for (int l1 = 0; l1 < 3; l1++)
    for (int l2 = 0; l2 < 3; l2++)
      for (int l3 = 0; l3 < 3; l3++)
        for (int l4 = 0; l4 < 3; l4++) c.push_back({om[l1], om[l2], om[l3], om[l4]});
  for (int l = 0; l < 3; l++)
    for (int m = 0; m < 3; m++) c.push_back({OP_P, om[l], OP_P, om[m]});
  for (int base : {OP_DX, OP_SSX, OP_XSX})
    for (int l1 = 0; l1 < 3; l1++)
      for (int l2 = 0; l2 < 3; l2++)
        for (int l3 = 0; l3 < 3; l3++)
          for (int l4 = 0; l4 < 3; l4++) c.push_back({base + l1, base + l2, base + l3, base + l4});
  for (int l = 0; l < 3; l++)
    for (int m = 0; m < 3; m++) c.push_back({OP_P, OP_DX + l, OP_P, OP_DX + m});
  return c;
}

const std::vector<std::array<int, 4>>& channels_table() {
  static const std::vector<std::array<int, 4>> t = make_channels();
  return t;
}

// Diquark matrices in the Dirac representation (gamma4 = diag(1,1,-1,-1),
// gamma_k = [[0, -i s_k], [i s_k, 0]], C = gamma4 gamma2), four non-zero
// entries each: C gamma_k = diag(s2 s_k, -s2 s_k), so
//   C gamma5       = diag(J, J), J = -i s2:  (0,1)=+1, (1,0)=-1, (2,3)=+1, (3,2)=-1
//   i C gamma_1    = diag(s3, -s3)
//   C gamma_2      = diag(1, -1)
//   -i C gamma_3   = diag(s1, -s1)
const int kGam[4][4][3] = {{{0, 1, +1}, {1, 0, -1}, {2, 3, +1}, {3, 2, -1}},
                           {{0, 0, +1}, {1, 1, -1}, {2, 2, -1}, {3, 3, +1}},
                           {{0, 0, +1}, {1, 1, +1}, {2, 2, -1}, {3, 3, -1}},
                           {{0, 1, +1}, {1, 0, +1}, {2, 3, -1}, {3, 2, -1}}};
// Permutations of three colours and their signs (eps tensor).
const int kEps[6][4] = {{0, 1, 2, +1}, {1, 2, 0, +1}, {2, 0, 1, +1},
                        {0, 2, 1, -1}, {2, 1, 0, -1}, {1, 0, 2, -1}};

bool is_strange(char f) { return f == 's'; }

// Family of a sink term, the slot order (Gamma pair, delta) in it and the
// sign of that order.  A family tensor takes eps over (Gamma pair, delta) in
// that order; the operator's eps runs over the quark string, so a term whose
// (gi, gj, dk) is an odd permutation of the string carries a sign -1 (the
// octet terms are all cyclic).  Renaming the two summed (spin, colour) pairs
// of a diquark gives D_sl[x, y] = -(Gamma1 symmetry) D_ls[y, x]: +D_ls[y, x]
// for C gamma5 (antisymmetric, like eps), -D_ls[y, x] for the symmetric
// eta_l C gamma_l, so an (s, l) diquark is read as (l, s) with its two slots
// swapped and that sign.
int perm_parity(const int* p, int n);
int family_of(const char* flav, const Term& t, int slots[3], int* sign) {
  bool a = is_strange(flav[t.gi]), b = is_strange(flav[t.gj]), c = is_strange(flav[t.dk]);
  slots[0] = t.gi; slots[1] = t.gj; slots[2] = t.dk;
  *sign = perm_parity(slots, 3);
  if (a && !b) {
    std::swap(a, b);
    std::swap(slots[0], slots[1]);
    if (t.g > 0) *sign = -*sign;
  }
  if (t.g == 0) {
    if (!a && !b) return c ? F_LLS : F_LLL;
    if (!a && b) return c ? F_LSS : F_LSL;
    return -1;  // (s, s) C gamma5 diquark: in no operator here
  }
  const int l = t.g - 1;
  if (!a && !b) return (c ? F_LLSV_X : F_LLLV_X) + l;
  if (!a && b) return (c ? F_LSSV_X : F_LSLV_X) + l;
  return (c ? F_SSS_X : F_SSLV_X) + l;
}

// Global tensor index and sign; families with two identical diquark quarks
// are stored with their first two indices ordered: symmetric under the
// exchange for C gamma5 (eps and C gamma5 both antisymmetric), antisymmetric
// for the symmetric vector matrices (zero at e0 = e1: returns -1).
int zindex(int fam, int a, int e0, int e1, int e2, int* sgn) {
  *sgn = 1;
  if (kFamSym[fam] > 0 && e1 < e0) std::swap(e0, e1);
  if (kFamSym[fam] < 0) {
    if (e0 == e1) return -1;
    if (e1 < e0) { std::swap(e0, e1); *sgn = -1; }
  }
  return (fam * 2 + a) * 1728 + e0 * 144 + e1 * 12 + e2;
}

struct SrcEntry { int eta[3]; int val; };

std::vector<SrcEntry> source_entries(const Term& t, int ext) {
  std::vector<SrcEntry> out;
  for (auto& e : kEps)
    for (auto& g : kGam[t.g]) {
      int sp[3];
      sp[t.gi] = g[0]; sp[t.gj] = g[1]; sp[t.dk] = ext;
      SrcEntry s;
      for (int m = 0; m < 3; m++) s.eta[m] = 3 * sp[m] + e[m];
      s.val = e[3] * g[2];
      out.push_back(s);
    }
  return out;
}

int perm_parity(const int* p, int n) {
  int inv = 0;
  for (int i = 0; i < n; i++)
    for (int j = i + 1; j < n; j++) inv += p[i] > p[j];
  return (inv & 1) ? -1 : 1;
}

using Row = std::vector<std::pair<int, int>>;  // (tensor index, weight), sorted

struct NatBlock {           // a block in the diagram's natural axis order
  std::vector<int> ext;     // source baryons (0 = B3, 1 = B4) whose spin it carries
  std::vector<int> osz;     // open axis sizes (diagram order)
  std::vector<Row> rows;    // index ((a * 2^next + ev) * K + ov)
};

int flat_open(const std::vector<int>& osz, const std::vector<int>& ov) {
  int f = 0;
  for (size_t i = 0; i < osz.size(); i++) f = f * osz[i] + ov[i];
  return f;
}
int flat_ext(const std::vector<int>& ev) {
  int f = 0;
  for (int v : ev) f = 2 * f + v;
  return f;
}

struct Variant {
  std::vector<int64_t> key;
  std::vector<int> pe, po;  // canonical axis i = natural axis pe[i] / po[i]
  int sgn;
};

Variant canonical(const NatBlock& b) {
  const int ne = (int)b.ext.size(), no = (int)b.osz.size();
  const int K = std::accumulate(b.osz.begin(), b.osz.end(), 1, std::multiplies<int>());
  std::vector<int> pe(ne), po(no);
  std::iota(pe.begin(), pe.end(), 0);
  Variant best;
  bool have = false;
  do {
    std::iota(po.begin(), po.end(), 0);
    do {
      for (int sgn : {1, -1}) {
        std::vector<int> oszc(no);
        for (int i = 0; i < no; i++) oszc[i] = b.osz[po[i]];
        std::vector<const Row*> crow(b.rows.size());
        // natural -> canonical
        for (int a = 0; a < 2; a++)
          for (int evf = 0; evf < (1 << ne); evf++)
            for (int ovf = 0; ovf < K; ovf++) {
              std::vector<int> ev(ne), ov(no);
              for (int i = ne - 1, x = evf; i >= 0; i--, x >>= 1) ev[i] = x & 1;
              for (int i = no - 1, x = ovf; i >= 0; i--) { ov[i] = x % b.osz[i]; x /= b.osz[i]; }
              std::vector<int> evc(ne), ovc(no);
              for (int i = 0; i < ne; i++) evc[i] = ev[pe[i]];
              for (int i = 0; i < no; i++) ovc[i] = ov[po[i]];
              int ci = (a * (1 << ne) + flat_ext(evc)) * K + flat_open(oszc, ovc);
              crow[ci] = &b.rows[(a * (1 << ne) + evf) * K + ovf];
            }
        std::vector<int64_t> key;
        key.push_back(ne);
        key.push_back(no);
        for (int v : oszc) key.push_back(v);
        for (const Row* r : crow) {
          key.push_back((int64_t)r->size());
          for (auto& zw : *r) { key.push_back(zw.first); key.push_back(sgn * zw.second); }
        }
        if (!have || key < best.key) { best.key = key; best.pe = pe; best.po = po; best.sgn = sgn; have = true; }
      }
    } while (std::next_permutation(po.begin(), po.end()));
  } while (std::next_permutation(pe.begin(), pe.end()));
  return best;
}

struct UBlock {
  int ne, no;
  std::vector<int> osz;     // canonical open sizes
  std::vector<Row> rows;    // canonical order
  int fam_mask = 0;
  int base = 0;
};

// Offset of a natural (a, ev, ov) entry of a block stored canonically.
int canon_offset(const UBlock& u, const Variant& v, int a, const std::vector<int>& ev,
                 const std::vector<int>& ov) {
  const int K = std::accumulate(u.osz.begin(), u.osz.end(), 1, std::multiplies<int>());
  std::vector<int> evc(u.ne), ovc(u.no);
  for (int i = 0; i < u.ne; i++) evc[i] = ev[v.pe[i]];
  for (int i = 0; i < u.no; i++) ovc[i] = ov[v.po[i]];
  return u.base + (a * (1 << u.ne) + flat_ext(evc)) * K + flat_open(u.osz, ovc);
}

}  // namespace

int channel_count() { return (int)channels_table().size(); }

void channel_names(int id, const char* out[4]) {
  const auto& c = channels_table()[id];
  for (int i = 0; i < 4; i++) out[i] = kOps[c[i]].name;
}

bool build_plan(const int* channels, int n, Plan* plan, std::string* err, int spin_offset) {
  const auto& table = channels_table();
  if (n <= 0) { *err = "empty channel list"; return false; }
  if (spin_offset != 0 && spin_offset != 2) { *err = "spin offset must be 0 or 2"; return false; }
  const int off = spin_offset;
  for (int i = 0; i < n; i++) {
    if (channels[i] < 0 || channels[i] >= (int)table.size()) { *err = "unknown channel id " + std::to_string(channels[i]); return false; }
    for (int j = 0; j < i; j++)
      if (channels[j] == channels[i]) { *err = "duplicate channel id " + std::to_string(channels[i]); return false; }
  }
  Plan P;
  P.channels.assign(channels, channels + n);
  P.spin_offset = off;

  std::map<std::vector<int64_t>, int> uniq;
  std::vector<UBlock> ublocks;
  // promA/promB: source baryons whose delta-quark minority enters that block as
  // a full (spin, colour) open index; the external spin then selects a slice
  // of it (Appendix A: a block with that quark's colour open and its spin
  // fixed is a sub-block of the one with both open).
  struct Inst {
    int ch_pos; double coef; int uA, uB; Variant vA, vB;
    std::vector<int> extA, extB, promA, promB, osz, oszA, oszB, open_k;
  };
  std::vector<Inst> insts;

  for (int cp = 0; cp < n; cp++) {
    const auto& ch = table[channels[cp]];
    const Op* op[4] = {&kOps[ch[0]], &kOps[ch[1]], &kOps[ch[2]], &kOps[ch[3]]};
    P.n_strange.push_back(op[0]->n_s + op[1]->n_s);
    char sinkf[6], srcf[6];
    for (int i = 0; i < 3; i++) {
      sinkf[i] = op[0]->flav[i]; sinkf[3 + i] = op[1]->flav[i];
      srcf[i] = op[2]->flav[i]; srcf[3 + i] = op[3]->flav[i];
    }
    for (int t3 = 0; t3 < op[2]->nterm; t3++)
      for (int t4 = 0; t4 < op[3]->nterm; t4++) {
        const Term src[2] = {op[2]->t[t3], op[3]->t[t4]};
        const double c34 = src[0].coef * src[1].coef * op[2]->scale * op[3]->scale;
        std::vector<int> seen;  // bitmask of S1 already classified
        int perm[6] = {0, 1, 2, 3, 4, 5};
        do {
          bool ok = true;
          for (int i = 0; i < 6 && ok; i++) ok = sinkf[i] == srcf[perm[i]];
          if (!ok) continue;
          int s1 = (1 << perm[0]) | (1 << perm[1]) | (1 << perm[2]);
          if (std::find(seen.begin(), seen.end(), s1) != seen.end()) continue;
          seen.push_back(s1);
          const int parity = perm_parity(perm, 6);
          // which block (0 = A at X+r, 1 = B at X) holds each source tensor
          int att[2], minority[2];
          for (int k = 0; k < 2; k++) {
            int inA = 0;
            for (int j = 3 * k; j < 3 * k + 3; j++) inA += (s1 >> j) & 1;
            att[k] = inA >= 2 ? 0 : 1;
            minority[k] = -1;
            for (int j = 3 * k; j < 3 * k + 3; j++) {
              bool in_att = (((s1 >> j) & 1) != 0) == (att[k] == 0);
              if (!in_att) minority[k] = j;
            }
          }
          std::vector<int> opens, osz;
          for (int k = 0; k < 2; k++)
            if (minority[k] >= 0) {
              opens.push_back(k);
              osz.push_back(minority[k] - 3 * k == src[k].dk ? 3 : 12);
            }
          const int K = std::accumulate(osz.begin(), osz.end(), 1, std::multiplies<int>());
          NatBlock nb[2];
          std::vector<int> prom[2];
          for (int blk = 0; blk < 2; blk++) {
            NatBlock& b = nb[blk];
            b.osz = osz;
            for (int k = 0; k < 2; k++) {
              int dpos = 3 * k + src[k].dk;
              const bool incoming_delta = att[k] != blk && minority[k] == dpos;
              if (incoming_delta) {
                prom[blk].push_back(k);
                for (size_t i = 0; i < opens.size(); i++)
                  if (opens[i] == k) b.osz[i] = 12;
                continue;
              }
              int carrier = (minority[k] != dpos) ? att[k] : 1 - att[k];
              if (carrier == blk) b.ext.push_back(k);
            }
            const Op* sink = op[blk];
            int pos[3];
            for (int s = 0; s < 3; s++) pos[s] = perm[3 * blk + s];
            // same-flavour permutations of the sink slots (with parity)
            std::vector<std::array<int, 4>> pis;
            int p3[3] = {0, 1, 2};
            do {
              if (sink->flav[p3[0]] == sink->flav[0] && sink->flav[p3[1]] == sink->flav[1] &&
                  sink->flav[p3[2]] == sink->flav[2])
                pis.push_back({p3[0], p3[1], p3[2], perm_parity(p3, 3)});
            } while (std::next_permutation(p3, p3 + 3));
            std::vector<int> attk;
            for (int k = 0; k < 2; k++)
              if (att[k] == blk) attk.push_back(k);
            const int ne = (int)b.ext.size();
            const int Kb = std::accumulate(b.osz.begin(), b.osz.end(), 1, std::multiplies<int>());
            b.rows.assign(2 * (1 << ne) * Kb, Row());
            for (int a = 0; a < 2; a++)
              for (int evf = 0; evf < (1 << ne); evf++)
                for (int ovf = 0; ovf < Kb; ovf++) {
                  int evk[2] = {-1, -1}, ovk[2] = {-1, -1};
                  for (int i = ne - 1, x = evf; i >= 0; i--, x >>= 1) evk[b.ext[i]] = x & 1;
                  for (int i = (int)opens.size() - 1, x = ovf; i >= 0; i--) { ovk[opens[i]] = x % b.osz[i]; x /= b.osz[i]; }
                  std::map<int, int> acc;
                  // enumerate entries of the attached tensors (at most two)
                  std::vector<std::vector<SrcEntry>> lists;
                  for (int k : attk) {
                    bool dmin = minority[k] >= 0 && minority[k] - 3 * k == src[k].dk;
                    // a delta minority leaves only its colour here (spin placeholder 0,
                    // filtered against the 3-valued open index below)
                    auto all = source_entries(src[k], dmin ? 0 : off + evk[k]);
                    std::vector<SrcEntry> keep;
                    for (auto& e : all)
                      if (minority[k] < 0 || e.eta[minority[k] - 3 * k] == ovk[k]) keep.push_back(e);
                    lists.push_back(keep);
                  }
                  size_t n0 = lists.size() > 0 ? lists[0].size() : 1;
                  size_t n1 = lists.size() > 1 ? lists[1].size() : 1;
                  for (size_t i0 = 0; i0 < n0; i0++)
                    for (size_t i1 = 0; i1 < n1; i1++) {
                      int eta[6] = {-1, -1, -1, -1, -1, -1};
                      int w = 1;
                      for (size_t li = 0; li < lists.size(); li++) {
                        const SrcEntry& e = lists[li][li == 0 ? i0 : i1];
                        int k = attk[li];
                        for (int m = 0; m < 3; m++) eta[3 * k + m] = e.eta[m];
                        w *= e.val;
                      }
                      for (int k = 0; k < 2; k++)
                        if (att[k] != blk && minority[k] >= 0) eta[minority[k]] = ovk[k];  // (spin, colour)
                      for (auto& pi : pis) {
                        int ein[3];
                        for (int s = 0; s < 3; s++) ein[s] = eta[pos[pi[s]]];
                        for (int t = 0; t < sink->nterm; t++) {
                          int sl[3], zs, fs;
                          int fam = family_of(sink->flav, sink->t[t], sl, &fs);
                          int z = zindex(fam, a, ein[sl[0]], ein[sl[1]], ein[sl[2]], &zs);
                          if (z >= 0) acc[z] += fs * zs * w * pi[3] * sink->t[t].coef;
                        }
                      }
                    }
                  Row& r = b.rows[(a * (1 << ne) + evf) * Kb + ovf];
                  for (auto& kv : acc)
                    if (kv.second != 0) r.push_back(kv);
                }
          }
          Inst in;
          in.ch_pos = cp;
          in.coef = parity * c34 * op[0]->scale * op[1]->scale;
          in.extA = nb[0].ext; in.extB = nb[1].ext; in.osz = osz;
          in.promA = prom[0]; in.promB = prom[1];
          in.open_k = opens;
          in.oszA = nb[0].osz; in.oszB = nb[1].osz;
          for (int blk = 0; blk < 2; blk++) {
            Variant v = canonical(nb[blk]);
            auto it = uniq.find(v.key);
            int id;
            if (it == uniq.end()) {
              id = (int)ublocks.size();
              uniq.emplace(v.key, id);
              UBlock u;
              const std::vector<int>& bosz = nb[blk].osz;
              u.ne = (int)nb[blk].ext.size();
              u.no = (int)bosz.size();
              u.osz.resize(u.no);
              for (int i = 0; i < u.no; i++) u.osz[i] = bosz[v.po[i]];
              const int Kc = std::accumulate(bosz.begin(), bosz.end(), 1, std::multiplies<int>());
              u.rows.assign(nb[blk].rows.size(), Row());
              for (int a = 0; a < 2; a++)
                for (int evf = 0; evf < (1 << u.ne); evf++)
                  for (int ovf = 0; ovf < Kc; ovf++) {
                    std::vector<int> ev(u.ne), ov(u.no);
                    for (int i = u.ne - 1, x = evf; i >= 0; i--, x >>= 1) ev[i] = x & 1;
                    for (int i = u.no - 1, x = ovf; i >= 0; i--) { ov[i] = x % bosz[i]; x /= bosz[i]; }
                    int ci = canon_offset(u, v, a, ev, ov);  // base 0 at this point
                    Row r = nb[blk].rows[(a * (1 << u.ne) + evf) * Kc + ovf];
                    for (auto& zw : r) { zw.second *= v.sgn; u.fam_mask |= 1 << (zw.first / kFamEntries); }
                    u.rows[ci] = r;
                  }
              ublocks.push_back(u);
            } else {
              id = it->second;
            }
            if (blk == 0) { in.uA = id; in.vA = v; } else { in.uB = id; in.vB = v; }
          }
          insts.push_back(in);
          DiagramInfo di{cp, t3, t4, K, parity, in.coef};
          P.diagrams.push_back(di);
        } while (std::next_permutation(perm, perm + 6));
      }
  }

  // --- group blocks by the families they read, assign row offsets ---------
  // group order: lll | lss | lsl | lsl+lls (the last two share slot 0) |
  // sss_x | sss_y | sss_z | per vector index l: lll_l | lsl_l+lls_l |
  // lss_l+ssl_l.  A block goes to the first group whose families cover the
  // ones it reads (a block of empty rows to lsl+lls).
  std::vector<std::array<int, 2>> gfam = {{F_LLL, -1},   {F_LSS, -1},   {F_LSL, -1},  {F_LSL, F_LLS},
                                          {F_SSS_X, -1}, {F_SSS_Y, -1}, {F_SSS_Z, -1}};
  for (int l = 0; l < 3; l++) {
    gfam.push_back({F_LLLV_X + l, -1});
    gfam.push_back({F_LSLV_X + l, F_LLSV_X + l});
    gfam.push_back({F_LSSV_X + l, F_SSLV_X + l});
  }
  std::vector<std::vector<int>> members(gfam.size());
  for (int u = 0; u < (int)ublocks.size(); u++) {
    const int m = ublocks[u].fam_mask;
    int g = m == 0 ? 3 : -1;
    for (size_t k = 0; k < gfam.size() && g < 0; k++) {
      const int cover = (1 << gfam[k][0]) | (gfam[k][1] >= 0 ? 1 << gfam[k][1] : 0);
      if ((m & ~cover) == 0) g = (int)k;
    }
    if (g < 0) { *err = "internal: block reads an unexpected family set"; return false; }
    members[g].push_back(u);
  }
  int row = 0;
  P.row_ptr.push_back(0);
  for (size_t g = 0; g < gfam.size(); g++) {
    if (members[g].empty()) continue;
    GroupInfo gi;
    gi.first_row = row;
    gi.fam[0] = gfam[g][0];
    gi.fam[1] = gfam[g][1];
    for (int u : members[g]) {
      UBlock& ub = ublocks[u];
      ub.base = row;
      for (auto& r : ub.rows) {
        for (auto& zw : r) {
          int fam = zw.first / kFamEntries, local = zw.first % kFamEntries;
          int slot = fam == gi.fam[0] ? 0 : 1;
          if (fam != gi.fam[slot]) { *err = "internal: family slot"; return false; }
          if (zw.second < -32768 || zw.second > 32767) { *err = "internal: weight range"; return false; }
          P.entries.push_back((uint32_t)(slot * kFamEntries + local) |
                              ((uint32_t)(uint16_t)(int16_t)zw.second << 16));
        }
        P.row_ptr.push_back((int)P.entries.size());
        row++;
      }
    }
    gi.n_rows = row - gi.first_row;
    P.groups.push_back(gi);
  }
  P.n_out = row;
  P.n_blocks = (int)ublocks.size();
  // the diquarks the groups' families need, in kind order
  {
    bool need[N_DIQUARK] = {false};
    for (const GroupInfo& gi : P.groups)
      for (int sl = 0; sl < 2; sl++)
        if (gi.fam[sl] >= 0) need[kFamDiquark[gi.fam[sl]]] = true;
    for (int d = 0; d < N_DIQUARK; d++)
      if (need[d]) P.diquarks.push_back(d);
  }
  // Compact shared-memory storage of the tensor entries: each group gets
  // positions for the entries its rows read; an entry the previous group left
  // in place (same family in the same slot) keeps its position, so it is
  // neither recomputed nor moved.  entries[] are rewritten to positions.
  {
    std::map<int, int> live;  // (slot * kFamEntries + local) -> position, valid for the current families
    int prev_fam[2] = {-1, -1};
    P.zneed_first.push_back(0);
    P.z_slots = 0;
    for (const GroupInfo& gi : P.groups) {
      // drop entries of a slot whose family changes
      for (int sl = 0; sl < 2; sl++)
        if (gi.fam[sl] != prev_fam[sl])
          for (auto it = live.begin(); it != live.end();) {
            if (it->first / kFamEntries == sl) it = live.erase(it);
            else ++it;
          }
      std::vector<char> used(8192, 0);
      for (auto& kv : live) used[kv.second] = 1;
      int next = 0;
      for (int r = gi.first_row; r < gi.first_row + gi.n_rows; r++)
        for (int k = P.row_ptr[r]; k < P.row_ptr[r + 1]; k++) {
          const int z = (int)(P.entries[k] & 0xffffu);
          auto it = live.find(z);
          int pos;
          if (it == live.end()) {
            while (next < 8192 && used[next]) next++;
            if (next >= 8192) { *err = "internal: tensor positions"; return false; }
            pos = next;
            used[pos] = 1;
            live.emplace(z, pos);
            const int sl = z / kFamEntries, local = z % kFamEntries;
            P.zneed.push_back((uint32_t)pos | ((uint32_t)sl << 13) | ((uint32_t)local << 14));
          } else {
            pos = it->second;
          }
          P.entries[k] = (P.entries[k] & 0xffff0000u) | (uint32_t)pos;
          P.z_slots = std::max(P.z_slots, pos + 1);
        }
      prev_fam[0] = gi.fam[0];
      prev_fam[1] = gi.fam[1];
      // The entries of a group are formed one per thread in list order; with
      // 16-byte entries (FP64, double-float) eight consecutive threads share a
      // wavefront.  Order the list so that each such eight differ, where they
      // can, in the bank group (mod 8) of the three shared-memory addresses a
      // thread touches: its diquark row (3 e01 + c2), its propagator row
      // (12 (3 a + c2) + e2) and its store position.
      {
        const size_t z0 = (size_t)P.zneed_first.back(), z1 = P.zneed.size();
        std::vector<uint32_t> rest(P.zneed.begin() + (long)z0, P.zneed.end());
        auto keys = [](uint32_t zn, int out[3]) {
          const int local = (int)(zn >> 14), pos = (int)(zn & 0x1fffu);
          const int a = local / 1728, e01 = (local % 1728) / 12, e2 = local % 12;
          out[0] = (3 * e01) & 7;
          out[1] = (36 * a + e2) & 7;
          out[2] = pos & 7;
        };
        size_t w = z0;
        while (!rest.empty()) {
          bool used[3][8] = {{false}};
          for (int lane = 0; lane < 8 && !rest.empty(); lane++) {
            size_t best = 0;
            int best_clash = 4;
            for (size_t j = 0; j < rest.size() && best_clash > 0; j++) {
              int k[3];
              keys(rest[j], k);
              const int clash = (int)used[0][k[0]] + (int)used[1][k[1]] + (int)used[2][k[2]];
              if (clash < best_clash) { best_clash = clash; best = j; }
            }
            int k[3];
            keys(rest[best], k);
            for (int m = 0; m < 3; m++) used[m][k[m]] = true;
            P.zneed[w++] = rest[best];
            rest.erase(rest.begin() + (long)best);
          }
        }
        if (w != z1) { *err = "internal: tensor entry order"; return false; }
      }
      P.zneed_first.push_back((int)P.zneed.size());
    }
  }

  // task products: one per aligned block pair, all 16 spin combinations.
  // Row rA enumerates (a, spins of extA, spins of promA); a promoted delta
  // minority of source baryon k is read at spin e_k of the 12-valued axis.
  {
    std::map<std::vector<int>, int> task_id;
    std::vector<std::vector<std::pair<int, double>>> tc(n * 16);
    for (const Inst& in : insts) {
      const UBlock& A = ublocks[in.uA];
      const UBlock& B = ublocks[in.uB];
      const int no = (int)in.osz.size();
      const int n1 = no > 0 ? in.osz[0] : 1, n2 = no > 1 ? in.osz[1] : 1;
      const int neA = (int)(in.extA.size() + in.promA.size()), neB = (int)(in.extB.size() + in.promB.size());
      PairTask t{};
      t.nA = 2 << neA;
      t.nB = 2 << neB;
      t.n1 = n1;
      t.n2 = n2;
      auto side_offset = [&](const UBlock& U, const Variant& v, const std::vector<int>& ext,
                             const std::vector<int>& prom, const std::vector<int>& bosz, int a, const int e[2],
                             int i, int j) {
        std::vector<int> ev;
        for (int k : ext) ev.push_back(e[k]);
        std::vector<int> ov;
        const int dv[2] = {i, j};
        for (int x = 0; x < no; x++) {
          int val = dv[x];
          if (bosz[x] != in.osz[x]) {
            // promoted axis (12 values in the block, 3 in the diagram): its
            // source baryon is the one in prom whose open axis this is
            int k = in.open_k[x];
            val = 3 * (off + e[k]) + dv[x];
          }
          ov.push_back(val);
        }
        return canon_offset(U, v, a, ev, ov);
      };
      auto decode = [](int r, const std::vector<int>& ext, const std::vector<int>& prom, int& a, int e[2]) {
        const int ne = (int)(ext.size() + prom.size());
        a = r >> ne;
        int x = r & ((1 << ne) - 1);
        for (int i = (int)prom.size() - 1; i >= 0; i--, x >>= 1) e[prom[i]] = x & 1;
        for (int i = (int)ext.size() - 1; i >= 0; i--, x >>= 1) e[ext[i]] = x & 1;
      };
      for (int rA = 0; rA < t.nA; rA++) {
        int a, e[2] = {0, 0};
        decode(rA, in.extA, in.promA, a, e);
        t.offA[rA] = side_offset(A, in.vA, in.extA, in.promA, in.oszA, a, e, 0, 0);
        if (rA == 0) {
          t.sA1 = n1 > 1 ? side_offset(A, in.vA, in.extA, in.promA, in.oszA, a, e, 1, 0) - t.offA[0] : 0;
          t.sA2 = n2 > 1 ? side_offset(A, in.vA, in.extA, in.promA, in.oszA, a, e, 0, 1) - t.offA[0] : 0;
        } else {
          // strides must not depend on the row (checked)
          const int s1 = n1 > 1 ? side_offset(A, in.vA, in.extA, in.promA, in.oszA, a, e, 1, 0) - t.offA[rA] : 0;
          const int s2 = n2 > 1 ? side_offset(A, in.vA, in.extA, in.promA, in.oszA, a, e, 0, 1) - t.offA[rA] : 0;
          if (s1 != t.sA1 || s2 != t.sA2) { *err = "internal: row-dependent stride"; return false; }
        }
      }
      for (int rB = 0; rB < t.nB; rB++) {
        int b, e[2] = {0, 0};
        decode(rB, in.extB, in.promB, b, e);
        t.offB[rB] = side_offset(B, in.vB, in.extB, in.promB, in.oszB, b, e, 0, 0);
        if (rB == 0) {
          t.sB1 = n1 > 1 ? side_offset(B, in.vB, in.extB, in.promB, in.oszB, b, e, 1, 0) - t.offB[0] : 0;
          t.sB2 = n2 > 1 ? side_offset(B, in.vB, in.extB, in.promB, in.oszB, b, e, 0, 1) - t.offB[0] : 0;
        } else {
          const int s1 = n1 > 1 ? side_offset(B, in.vB, in.extB, in.promB, in.oszB, b, e, 1, 0) - t.offB[rB] : 0;
          const int s2 = n2 > 1 ? side_offset(B, in.vB, in.extB, in.promB, in.oszB, b, e, 0, 1) - t.offB[rB] : 0;
          if (s1 != t.sB1 || s2 != t.sB2) { *err = "internal: row-dependent stride"; return false; }
        }
      }
      // The product sums over both open axes, so listing them in the other
      // order gives the same task: put them in a canonical order before the
      // identical tasks are merged (the diagrams of one block pair often
      // meet the two open indices in opposite orders).
      if (std::tie(t.n2, t.sA2, t.sB2) > std::tie(t.n1, t.sA1, t.sB1)) {
        std::swap(t.n1, t.n2);
        std::swap(t.sA1, t.sA2);
        std::swap(t.sB1, t.sB2);
      }
      std::vector<int> key = {t.nA, t.nB, t.n1, t.n2, t.sA1, t.sA2, t.sB1, t.sB2};
      for (int r = 0; r < t.nA; r++) key.push_back(t.offA[r]);
      for (int r = 0; r < t.nB; r++) key.push_back(t.offB[r]);
      auto it = task_id.find(key);
      int id;
      if (it == task_id.end()) {
        id = (int)P.tasks.size();
        task_id.emplace(key, id);
        P.tasks.push_back(t);
      } else {
        id = it->second;
      }
      for (int s = 0; s < 16; s++) {
        int a = s & 1, b = (s >> 1) & 1, e[2] = {(s >> 2) & 1, (s >> 3) & 1};
        int rA = a, rB = b;
        for (int k : in.extA) rA = 2 * rA + e[k];
        for (int k : in.promA) rA = 2 * rA + e[k];
        for (int k : in.extB) rB = 2 * rB + e[k];
        for (int k : in.promB) rB = 2 * rB + e[k];
        tc[in.ch_pos * 16 + s].push_back({id * 16 + rA * t.nB + rB, in.coef * in.vA.sgn * in.vB.sgn});
      }
    }
    P.tcontrib_ptr.push_back(0);
    for (auto& c : tc) {
      std::map<int, double> m;
      for (auto& p : c) m[p.first] += p.second;
      for (auto& kv : m)
        if (kv.second != 0.0) { P.tcontrib_item.push_back(kv.first); P.tcontrib_coef.push_back(kv.second); }
      P.tcontrib_ptr.push_back((int)P.tcontrib_item.size());
    }
  }

  // Products that vanish for every q: at each open-index step one of the two
  // rows has no terms (its weights cancelled), so it is exactly zero.  Their
  // contributions are dropped, and so are tasks none of whose products is
  // still read (all of them vanish, or the channels' sums cancelled them).
  {
    std::vector<char> empty_row(P.n_out);
    for (int r = 0; r < P.n_out; r++) empty_row[r] = P.row_ptr[r + 1] == P.row_ptr[r];
    const int nt = (int)P.tasks.size();
    std::vector<char> zero_prod((size_t)nt * 16, 1);
    for (int t = 0; t < nt; t++) {
      const PairTask& k = P.tasks[t];
      for (int ra = 0; ra < k.nA; ra++)
        for (int rb = 0; rb < k.nB; rb++) {
          bool z = true;
          for (int i1 = 0; i1 < k.n1 && z; i1++)
            for (int i2 = 0; i2 < k.n2 && z; i2++)
              z = empty_row[k.offA[ra] + i1 * k.sA1 + i2 * k.sA2] || empty_row[k.offB[rb] + i1 * k.sB1 + i2 * k.sB2];
          zero_prod[(size_t)t * 16 + ra * k.nB + rb] = z;
        }
    }
    std::vector<char> used(nt, 0);
    for (int it : P.tcontrib_item)
      if (!zero_prod[it]) used[it / 16] = 1;
    std::vector<int> new_id(nt, -1);
    std::vector<PairTask> kept;
    for (int t = 0; t < nt; t++)
      if (used[t]) {
        new_id[t] = (int)kept.size();
        kept.push_back(P.tasks[t]);
      }
    std::vector<int> ptr(1, 0), item;
    std::vector<double> coef;
    for (size_t o = 0; o + 1 < P.tcontrib_ptr.size(); o++) {
      for (int c = P.tcontrib_ptr[o]; c < P.tcontrib_ptr[o + 1]; c++) {
        const int it = P.tcontrib_item[c];
        if (zero_prod[it]) continue;
        item.push_back(new_id[it / 16] * 16 + it % 16);
        coef.push_back(P.tcontrib_coef[c]);
      }
      ptr.push_back((int)item.size());
    }
    P.tasks.swap(kept);
    P.tcontrib_ptr.swap(ptr);
    P.tcontrib_item.swap(item);
    P.tcontrib_coef.swap(coef);
  }

  P.pair_macs = 0;
  for (const PairTask& t : P.tasks) P.pair_macs += 16LL * t.n1 * t.n2;
  // bounds of every device table index (checked once on the host so that no
  // kernel can read outside a block row or the product buffer)
  for (const PairTask& t : P.tasks) {
    if (!((t.nA == 2 && t.nB == 8) || (t.nA == 4 && t.nB == 4) || (t.nA == 8 && t.nB == 2)) || t.n1 < 1 ||
        t.n2 < 1 || t.n1 * t.n2 > 0xffff) {
      *err = "internal: task shape";
      return false;
    }
    for (int r = 0; r < t.nA; r++)
      if (t.offA[r] < 0 || t.offA[r] + (t.n1 - 1) * t.sA1 + (t.n2 - 1) * t.sA2 >= P.n_out) { *err = "internal: task A range"; return false; }
    for (int r = 0; r < t.nB; r++)
      if (t.offB[r] < 0 || t.offB[r] + (t.n1 - 1) * t.sB1 + (t.n2 - 1) * t.sB2 >= P.n_out) { *err = "internal: task B range"; return false; }
    // strides are packed two per 32-bit word on the device (sA1 | sA2 << 16)
    if (t.sA1 < 0 || t.sA2 < 0 || t.sB1 < 0 || t.sB2 < 0 || t.sA1 > 0xffff || t.sA2 > 0xffff || t.sB1 > 0xffff ||
        t.sB2 > 0xffff) {
      *err = "internal: task stride";
      return false;
    }
  }
  for (int id : P.tcontrib_item)
    if (id < 0 || id >= 16 * (int)P.tasks.size()) { *err = "internal: task contribution index"; return false; }
  for (uint32_t e : P.entries)
    if ((int)(e & 0xffffu) >= P.z_slots) { *err = "internal: tensor position"; return false; }
  for (uint32_t z : P.zneed)
    if ((int)(z & 0x1fffu) >= P.z_slots || (z >> 14) >= (uint32_t)kFamEntries) { *err = "internal: tensor entry"; return false; }
  if ((int)P.row_ptr.size() != P.n_out + 1) { *err = "internal: row table"; return false; }
  // lane-interleaved 32-row chunks of every group (the build kernel's layout)
  P.chunk_first.assign(1, 0);
  for (const GroupInfo& g : P.groups) {
    for (int c0 = 0; c0 < g.n_rows; c0 += 32) {
      const int r0 = g.first_row + c0, nr = std::min(32, g.n_rows - c0);
      int len = 0;
      for (int l = 0; l < nr; l++) len = std::max(len, P.row_ptr[r0 + l + 1] - P.row_ptr[r0 + l]);
      const int base = (int)P.ell.size();
      P.ell.resize(P.ell.size() + (size_t)32 * len, 0u);  // weight 0, position 0
      // A row's terms may be summed in any order: at every step k, give each
      // lane a term whose tensor position falls in a bank group that no other
      // lane of its wavefront uses at that step, where it can.  The tables
      // serve the FP64 and double-float builds: a 16-byte entry spans four of
      // the 32 banks, so a 128-byte wavefront serves eight lanes and the bank
      // group is the position mod 8.
      constexpr int kLanes = 8, kGroups = 8;
      std::vector<std::vector<uint32_t>> left(nr);
      for (int l = 0; l < nr; l++)
        left[l].assign(P.entries.begin() + P.row_ptr[r0 + l], P.entries.begin() + P.row_ptr[r0 + l + 1]);
      for (int k = 0; k < len; k++)
        for (int h = 0; h < 32; h += kLanes) {
          bool used[kGroups] = {false};
          for (int l = h; l < std::min(nr, h + kLanes); l++) {
            std::vector<uint32_t>& v = left[l];
            if (v.empty()) continue;
            size_t pick = 0;
            for (size_t j = 0; j < v.size(); j++)
              if (!used[(v[j] & 0xffffu) % kGroups]) { pick = j; break; }
            used[(v[pick] & 0xffffu) % kGroups] = true;
            P.ell[base + 32 * k + l] = v[pick];
            v.erase(v.begin() + (long)pick);
          }
        }
      // then exchanges of two steps of one lane (terms or padding) while the
      // modelled shared-memory wavefronts of the two steps drop: distinct
      // positions in one bank group serialise, equal ones broadcast, padding
      // (weight 0) reads position 0
      auto group_cost = [&](int k, int h) {
        int cnt[kGroups] = {0}, seen[kGroups][kLanes], m = 0;
        for (int l = h; l < std::min(nr, h + kLanes); l++) {
          const uint32_t e = P.ell[base + 32 * k + l];
          const int pos = (int)(e & 0xffffu), b = pos % kGroups;
          bool dup = false;
          for (int j = 0; j < cnt[b]; j++) dup |= seen[b][j] == pos;
          if (!dup && cnt[b] < kLanes) {
            seen[b][cnt[b]++] = pos;
            m = std::max(m, cnt[b]);
          }
        }
        return m;
      };
      for (int sweep = 0; sweep < 4; sweep++) {
        bool improved = false;
        for (int l = 0; l < nr; l++)
          for (int k1 = 0; k1 < len; k1++)
            for (int k2 = k1 + 1; k2 < len; k2++) {
              uint32_t& a = P.ell[base + 32 * k1 + l];
              uint32_t& b = P.ell[base + 32 * k2 + l];
              if (a == b) continue;
              const int h = l / kLanes * kLanes;
              const int before = group_cost(k1, h) + group_cost(k2, h);
              std::swap(a, b);
              if (group_cost(k1, h) + group_cost(k2, h) < before) improved = true;
              else std::swap(a, b);
            }
        if (!improved) break;
      }
      P.ell_chunk.push_back({base, len});
    }
    P.chunk_first.push_back((int)P.ell_chunk.size());
  }
  for (const auto& c : P.ell_chunk)
    if (c.first < 0 || c.second < 0 || (size_t)c.first + 32 * (size_t)c.second > P.ell.size()) {
      *err = "internal: row chunk";
      return false;
    }
  for (uint32_t e : P.ell)
    if ((int)(e & 0xffffu) >= P.z_slots) { *err = "internal: tensor position"; return false; }
  if (P.groups.size() > (size_t)kMaxGroups) { *err = "internal: group count"; return false; }
  *plan = std::move(P);
  return true;
}

void make_batches(const Plan& plan, std::vector<Batch>* batches) {
  std::map<std::array<int, 3>, std::vector<int>> cls;
  for (int t = 0; t < (int)plan.tasks.size(); t++) {
    const PairTask& k = plan.tasks[t];
    cls[{k.nA, k.nB, k.n1 * k.n2}].push_back(t);
  }
  batches->clear();
  for (auto& kv : cls)
    for (size_t i = 0; i < kv.second.size(); i += 32) {
      Batch b;
      b.nA = kv.first[0];
      for (size_t j = i; j < kv.second.size() && j < i + 32; j++) b.tasks.push_back(kv.second[j]);
      batches->push_back(b);
    }
}

void make_units(const Plan& plan, const std::vector<Batch>& batches, int warps, int chunk, std::vector<int>* warp_ptr,
                std::vector<BatchUnit>* units) {
  if (chunk <= 0) {
    // contiguous split: the batches' open-index steps laid end to end and cut
    // into `warps` pieces of equal modelled cost, so every warp flushes its
    // products about once per batch it touches
    std::vector<long long> per_k(batches.size());
    long long total = 0;
    for (size_t b = 0; b < batches.size(); b++) {
      const PairTask& t = plan.tasks[batches[b].tasks[0]];
      per_k[b] = 128 + 4 * (t.nA + t.nB);
      total += per_k[b] * t.n1 * t.n2;
    }
    warp_ptr->assign(1, 0);
    units->clear();
    long long done = 0;
    size_t b = 0;
    int k = 0;
    for (int w = 0; w < warps; w++) {
      const long long target = total * (w + 1) / warps;
      while (b < batches.size() && done < target) {
        const PairTask& t = plan.tasks[batches[b].tasks[0]];
        const int K = t.n1 * t.n2;
        long long take = (target - done + per_k[b] - 1) / per_k[b];  // steps to reach the target
        if (w == warps - 1) take = K - k;
        const int k1 = (int)std::min<long long>(K, k + std::max<long long>(1, take));
        units->push_back(BatchUnit{(int)b, 0, k, k1});
        done += per_k[b] * (k1 - k);
        k = k1;
        if (k == K) { b++; k = 0; }
      }
      warp_ptr->push_back((int)units->size());
    }
    return;
  }
  std::vector<BatchUnit> all;
  for (int id = 0; id < (int)batches.size(); id++) {
    const PairTask& t = plan.tasks[batches[id].tasks[0]];
    const int K = t.n1 * t.n2;
    const int step = K > chunk ? chunk : K;
    for (int k = 0; k < K; k += step) all.push_back(BatchUnit{id, 0, k, std::min(K, k + step)});
  }
  auto cost = [&](const BatchUnit& u) {
    const Batch& b = batches[u.batch];
    const int nB = 16 / b.nA;
    return (long long)(u.k1 - u.k0) * (128 + 4 * (b.nA + nB)) + 128;
  };
  std::stable_sort(all.begin(), all.end(), [&](const BatchUnit& a, const BatchUnit& b) { return cost(a) > cost(b); });
  std::vector<long long> load(warps, 0);
  std::vector<std::vector<BatchUnit>> per(warps);
  for (const BatchUnit& u : all) {
    int best = 0;
    for (int w = 1; w < warps; w++)
      if (load[w] < load[best]) best = w;
    load[best] += cost(u);
    per[best].push_back(u);
  }
  warp_ptr->assign(1, 0);
  units->clear();
  for (auto& v : per) {
    for (auto& u : v) units->push_back(u);
    warp_ptr->push_back((int)units->size());
  }
}

namespace {

// Exact bank model of the fused products' 128-bit shared-memory loads.
struct BankModel {
  const Plan& p;
  std::vector<int> seg_of_row;  // n_out
  std::vector<int> res;         // shift residue (mod 8) per segment
  std::vector<int> shift;       // non-decreasing shifts with those residues
  // per task: rows read at (k, operand row), A rows then B rows: [K][nA + nB]
  std::vector<std::vector<int>> rows, slots;

  void init_rows() {
    rows.resize(p.tasks.size());
    for (size_t ti = 0; ti < p.tasks.size(); ti++) {
      const PairTask& t = p.tasks[ti];
      std::vector<int>& v = rows[ti];
      for (int i1 = 0; i1 < t.n1; i1++)
        for (int i2 = 0; i2 < t.n2; i2++) {
          for (int r = 0; r < t.nA; r++) v.push_back(t.offA[r] + i1 * t.sA1 + i2 * t.sA2);
          for (int r = 0; r < t.nB; r++) v.push_back(t.offB[r] + i1 * t.sB1 + i2 * t.sB2);
        }
    }
  }
  void update_shifts() {
    shift.assign(res.size(), 0);
    for (size_t s = 0; s < res.size(); s++) {
      const int prev = s ? shift[s - 1] : 0;
      shift[s] = prev + (((res[s] - prev) % 8) + 8) % 8;
    }
    slots.resize(rows.size());
    for (size_t ti = 0; ti < rows.size(); ti++) {
      slots[ti].resize(rows[ti].size());
      for (size_t j = 0; j < rows[ti].size(); j++) slots[ti][j] = rows[ti][j] + shift[seg_of_row[rows[ti][j]]];
    }
  }
  int slot(int row) const { return row + shift[seg_of_row[row]]; }
  // wavefronts of lanes [l0, l1) (one phase) of a batch over every load
  long long phase_cost(const std::vector<int>& tasks, int l0, int l1) const {
    if (l0 >= l1) return 0;
    const size_t n = slots[tasks[l0]].size();
    const int* sl[8];
    const int nl = l1 - l0;
    for (int l = 0; l < nl; l++) sl[l] = slots[tasks[l0 + l]].data();
    long long w = 0;
    for (size_t j = 0; j < n; j++) {
      int cnt[8] = {0, 0, 0, 0, 0, 0, 0, 0}, m = 0;
      for (int l = 0; l < nl; l++) {
        const int a = sl[l][j];
        bool dup = false;
        for (int i = 0; i < l; i++) dup |= sl[i][j] == a;
        if (!dup) m = std::max(m, ++cnt[a & 7]);
      }
      w += m;
    }
    return w;
  }
};

}  // namespace

void optimise_fused_layout(const Plan& plan, std::vector<Batch>* batches, FusedLayout* out) {
  const int n_out = plan.n_out;
  BankModel m{plan, std::vector<int>(n_out, 0), {}, {}, {}, {}};
  m.init_rows();
  // operand segments: merged row spans of every task side
  std::vector<std::pair<int, int>> span;
  for (size_t ti = 0; ti < plan.tasks.size(); ti++) {
    const PairTask& t = plan.tasks[ti];
    const std::vector<int>& v = m.rows[ti];
    for (int side = 0; side < 2; side++) {
      int lo = n_out, hi = -1;
      const int nr = t.nA + t.nB, r0 = side ? t.nA : 0, r1 = side ? nr : t.nA;
      for (size_t j = 0; j < v.size(); j++) {
        const int r = (int)(j % nr);
        if (r < r0 || r >= r1) continue;
        lo = std::min(lo, v[j]);
        hi = std::max(hi, v[j]);
      }
      if (hi >= 0) span.push_back({lo, hi});
    }
  }
  std::sort(span.begin(), span.end());
  std::vector<int> seg_first(1, 0);
  int end = -1;
  for (const auto& sp : span) {
    if (sp.first > end && sp.first > 0 && sp.first != seg_first.back()) seg_first.push_back(sp.first);
    end = std::max(end, sp.second);
  }
  for (size_t s = 0; s < seg_first.size(); s++) {
    const int e = s + 1 < seg_first.size() ? seg_first[s + 1] : n_out;
    for (int r = seg_first[s]; r < e; r++) m.seg_of_row[r] = (int)s;
  }
  m.res.assign(seg_first.size(), 0);
  m.update_shifts();
  // phases: (batch, first lane); cost cache
  auto phase_end = [&](int b, int p0) { return std::min((int)(*batches)[b].tasks.size(), p0 + 8); };
  auto total = [&]() {
    long long w = 0;
    for (int b = 0; b < (int)batches->size(); b++)
      for (int p0 = 0; p0 < (int)(*batches)[b].tasks.size(); p0 += 8) w += m.phase_cost((*batches)[b].tasks, p0, phase_end(b, p0));
    return w;
  };
  // batches of one class (same nA and open-index length) may trade tasks
  std::map<std::pair<int, int>, std::vector<int>> cls;
  for (int i = 0; i < (int)batches->size(); i++) {
    const PairTask& t = plan.tasks[(*batches)[i].tasks[0]];
    cls[{t.nA, t.n1 * t.n2}].push_back(i);
  }
  long long best = total();
  // segments each task reads.  A residue change of segment s moves later
  // segments by multiples of 8 only (same bank groups; segments never share
  // an address), so a trial on s re-costs just the phases that read s.
  std::vector<std::vector<char>> task_reads(plan.tasks.size(), std::vector<char>(seg_first.size(), 0));
  for (size_t ti = 0; ti < plan.tasks.size(); ti++)
    for (int r : m.rows[ti]) task_reads[ti][m.seg_of_row[r]] = 1;
  for (int sweep = 0; sweep < 3; sweep++) {
    bool improved = false;
    for (size_t s = 0; s < m.res.size(); s++) {  // segment shifts, one at a time
      std::vector<std::pair<int, int>> touched;  // phases reading segment s
      long long old_cost = 0;
      for (int b = 0; b < (int)batches->size(); b++) {
        const std::vector<int>& T = (*batches)[b].tasks;
        for (int p0 = 0; p0 < (int)T.size(); p0 += 8) {
          bool hit = false;
          for (int l = p0; l < phase_end(b, p0); l++) hit |= task_reads[T[l]][s] != 0;
          if (!hit) continue;
          touched.push_back({b, p0});
          old_cost += m.phase_cost(T, p0, phase_end(b, p0));
        }
      }
      int keep = m.res[s];
      long long keep_cost = old_cost;
      for (int v = 0; v < 8; v++) {
        if (v == m.res[s]) continue;
        const int saved = m.res[s];
        m.res[s] = v;
        m.update_shifts();
        long long w = 0;
        for (const auto& ph : touched) w += m.phase_cost((*batches)[ph.first].tasks, ph.second, phase_end(ph.first, ph.second));
        if (w < keep_cost) { keep_cost = w; keep = v; }
        m.res[s] = saved;
      }
      if (keep_cost < old_cost) { best += keep_cost - old_cost; improved = true; }
      m.res[s] = keep;
      m.update_shifts();
    }
    for (auto& kv : cls) {  // pairwise exchanges of lanes in different phases
      std::vector<std::pair<int, int>> pos;  // (batch, lane)
      std::map<std::pair<int, int>, long long> cost, ideal;
      for (int b : kv.second) {
        const std::vector<int>& T = (*batches)[b].tasks;
        for (int l = 0; l < (int)T.size(); l++) pos.push_back({b, l});
        for (int p0 = 0; p0 < (int)T.size(); p0 += 8) {
          cost[{b, p0}] = m.phase_cost(T, p0, phase_end(b, p0));
          ideal[{b, p0}] = (long long)m.slots[T[p0]].size();
        }
      }
      for (size_t i = 0; i < pos.size(); i++)
        for (size_t j = i + 1; j < pos.size(); j++) {
          const int b1 = pos[i].first, l1 = pos[i].second, b2 = pos[j].first, l2 = pos[j].second;
          const int p1 = l1 / 8 * 8, p2 = l2 / 8 * 8;
          if (b1 == b2 && p1 == p2) continue;
          const std::pair<int, int> k1{b1, p1}, k2{b2, p2};
          if (cost[k1] == ideal[k1] && cost[k2] == ideal[k2]) continue;  // both conflict-free already
          std::vector<int>& T1 = (*batches)[b1].tasks;
          std::vector<int>& T2 = (*batches)[b2].tasks;
          std::swap(T1[l1], T2[l2]);
          const long long c1 = m.phase_cost(T1, p1, phase_end(b1, p1)), c2 = m.phase_cost(T2, p2, phase_end(b2, p2));
          if (c1 + c2 < cost[k1] + cost[k2]) {
            best += c1 + c2 - cost[k1] - cost[k2];
            cost[k1] = c1;
            cost[k2] = c2;
            improved = true;
          } else {
            std::swap(T1[l1], T2[l2]);
          }
        }
    }
    if (!improved) break;
  }
  out->row_slot.resize(n_out);
  for (int r = 0; r < n_out; r++) out->row_slot[r] = m.slot(r);
  out->n_slots = n_out + (m.shift.empty() ? 0 : m.shift.back());
  out->wavefronts = best;
  long long ideal = 0;
  for (const Batch& b : *batches) ideal += (long long)m.slots[b.tasks[0]].size() * (((int)b.tasks.size() + 7) / 8);
  out->ideal = ideal;
}

void make_task_groups(const Plan& plan, int groups, std::vector<int>* group_ptr, std::vector<int>* group_task,
                      bool by_shape) {
  auto cost = [&](int t) {
    const PairTask& k = plan.tasks[t];
    return (long long)k.n1 * k.n2 * (4 * k.nA * k.nB + 2 * (k.nA + k.nB)) + 64;  // FMAs + loads + stores
  };
  // classes of tasks that share a code path (all tasks, or one class per nA)
  std::map<int, std::vector<int>> cls;
  for (int t = 0; t < (int)plan.tasks.size(); t++) cls[by_shape ? plan.tasks[t].nA : 0].push_back(t);
  long long total = 0;
  for (int t = 0; t < (int)plan.tasks.size(); t++) total += cost(t);
  group_ptr->assign(1, 0);
  group_task->clear();
  int left = groups;
  size_t ci = 0;
  for (auto& kv : cls) {
    long long ccost = 0;
    for (int t : kv.second) ccost += cost(t);
    // groups for this class in proportion to its cost (at least one each)
    const int remaining_classes = (int)(cls.size() - ci);
    int g = ci + 1 == cls.size() ? left : (int)std::max<long long>(1, (long long)groups * ccost / std::max(total, 1LL));
    g = std::min(g, left - (remaining_classes - 1));
    left -= g;
    ci++;
    std::vector<int> order = kv.second;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cost(a) > cost(b); });
    std::vector<long long> load(g, 0);
    std::vector<std::vector<int>> per(g);
    for (int t : order) {
      int best = 0;
      for (int i = 1; i < g; i++)
        if (load[i] < load[best]) best = i;
      load[best] += cost(t);
      per[best].push_back(t);
    }
    for (auto& v : per) {
      std::sort(v.begin(), v.end());
      for (int t : v) group_task->push_back(t);
      group_ptr->push_back((int)group_task->size());
    }
  }
}

}  // namespace bbc
