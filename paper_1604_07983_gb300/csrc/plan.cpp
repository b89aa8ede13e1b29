// plan.cpp -- host channel compiler (Sec. 4 (ii)-(iii) of arXiv:1604.07983).
//
// For every requested channel <B1 B2 | B3bar B4bar> it enumerates the Wick
// contractions of Eq. (2.4) grouped into the effective-block terms of
// Eq. (2.7), and packs, per term, the gathers that build the two effective
// blocks in momentum space from the stored baryon blocks.
//
// Stored blocks ("field blocks").  For a sink field B with flavour content
// sorted as u < d < s ("canonical positions" 0, 1, 2) the device stores
//
//   FB^B_alpha(x; y0, y1, y2) = sum_{monomials m} c_m sum_tau sign(tau)
//                                 N^m_alpha(x; y_tau(1), y_tau(2), y_tau(3)),
//
// tau assigning sink quark k of m to the canonical position of its flavour,
// N^m the normal block of Eq. (4.1).  With u = d (the isospin limit of
// Sec. 4 (i)) n shares p's storage, Sigma- shares Sigma+'s and Xi- shares
// Xi0's, up to an argument permutation and a sign found by comparing the
// symbolic expansions; two positions of equal flavour make FB antisymmetric
// (or, for Lambda / Sigma0 under u <-> d, symmetric), and such pairs are
// stored once.
//
// Effective blocks.  For source monomials (m3, m4) and the set S of source
// slots feeding B1, every permutation with P({1,2,3}) = S has sign
// sign(P0_S) sign(tau1) sign(tau2), so the B1 side of the term is
// sign(rho) FB^{B1}(source indices of S in canonical order), rho the
// flavour-preserving map from canonical positions to the sorted slots of S.
// The source tensor eps eps (Cg5)(Cg5) delta delta is split: each source
// baryon's eps and Cg5 go to the side holding two or three of its slots, its
// projector to the side of its third slot; indices of one side's slots that
// appear in a factor of the other side are the shared indices xi~ (Sec. 4
// (ii); for <p Lambda | p Xu> they are the six sets the paper lists).
#include "plan.h"

#include <algorithm>
#include <array>
#include <cmath>
#include <map>
#include <sstream>

namespace nbs {

namespace {

const double kR6 = 1.0 / std::sqrt(6.0);
const double kR2 = 1.0 / std::sqrt(2.0);

// C gamma5 in the Dirac representation (C = gamma4 gamma2)
const int kCG5[4][4] = {{0, 1, 0, 0}, {-1, 0, 0, 0}, {0, 0, 0, 1}, {0, 0, -1, 0}};

int eps3(int a, int b, int c) {
  if (a == b || b == c || a == c) return 0;
  // (a, b, c) is a permutation of (0, 1, 2)
  int inv = (a > b) + (a > c) + (b > c);
  return (inv & 1) ? -1 : 1;
}

int perm_sign(const int* p, int n) {
  int inv = 0;
  for (int i = 0; i < n; ++i)
    for (int j = i + 1; j < n; ++j) inv += p[i] > p[j];
  return (inv & 1) ? -1 : 1;
}

const int kPerm3[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};

using RKey = std::array<int, 4>;  // pattern, a0, a1, a2
using Recipe = std::map<RKey, double>;

// propagator index of a quark flavour: l = u = d and s for nflav = 2, u, d, s for 3
int lflav(int q, int nflav) { return nflav == 2 ? (q == FS ? 1 : 0) : q; }

int diquark_index(int nflav, int f0, int f1) {
  for (int d = 0; d < n_diquarks(nflav); ++d) {
    int g0, g1;
    diquark_flavours(nflav, d, g0, g1);
    if (g0 == f0 && g1 == f1) return d;
  }
  return -1;
}

// the pattern's diquark has two quarks of one flavour (symmetric in its two arguments)
bool same_flavour_diquark(int pat, int nflav) {
  int f0, f1;
  diquark_flavours(nflav, pat / nflav, f0, f1);
  return f0 == f1;
}

bool add_term(Recipe& R, int nflav, int f0, int f1, int f2, int a0, int a1, int a2, double c) {
  // N^{f0 f1 f2}(j_a0, j_a1, j_a2) = N^{f1 f0 f2}(j_a1, j_a0, j_a2)  (eps and Cg5 both antisymmetric)
  if (f0 > f1) { std::swap(f0, f1); std::swap(a0, a1); }
  const int d = diquark_index(nflav, f0, f1);
  if (d < 0) return false;  // two strange quarks in the diquark: not an octet field
  const int pat = d * nflav + f2;
  if (f0 == f1 && a0 > a1) std::swap(a0, a1);
  R[{pat, a0, a1, a2}] += c;
  return true;
}

void prune(Recipe& R) {
  for (auto it = R.begin(); it != R.end();) {
    if (std::fabs(it->second) < 1e-13) it = R.erase(it); else ++it;
  }
}

// R o pi : j -> FB(j_pi(0), j_pi(1), j_pi(2))
Recipe compose(const Recipe& R, const int* pi, int nflav) {
  Recipe out;
  for (auto& kv : R) {
    int pat = kv.first[0];
    int a0 = pi[kv.first[1]], a1 = pi[kv.first[2]], a2 = pi[kv.first[3]];
    if (same_flavour_diquark(pat, nflav) && a0 > a1) std::swap(a0, a1);
    out[{pat, a0, a1, a2}] += kv.second;
  }
  prune(out);
  return out;
}

bool equal_scaled(const Recipe& A, const Recipe& B, double s) {
  if (A.size() != B.size()) return false;
  for (auto& kv : A) {
    auto it = B.find(kv.first);
    if (it == B.end() || std::fabs(kv.second - s * it->second) > 1e-12) return false;
  }
  return true;
}

void canonical_flavours(int field, int cf[3]) {
  const Mono& m = field_monomials(field)[0];
  int q[3] = {m.q[0], m.q[1], m.q[2]};
  std::sort(q, q + 3);
  cf[0] = q[0]; cf[1] = q[1]; cf[2] = q[2];
}

bool field_recipe(int field, Recipe& R, int nflav) {
  int cf[3];
  canonical_flavours(field, cf);
  for (const Mono& m : field_monomials(field)) {
    for (auto& tau : kPerm3) {
      if (m.q[0] != cf[tau[0]] || m.q[1] != cf[tau[1]] || m.q[2] != cf[tau[2]]) continue;
      double c = m.c * perm_sign(tau, 3);
      if (!add_term(R, nflav, lflav(m.q[0], nflav), lflav(m.q[1], nflav), lflav(m.q[2], nflav), tau[0], tau[1], tau[2],
                    c))
        return false;
    }
  }
  prune(R);
  return true;
}

struct FieldMap { int type = -1; int pi[3] = {0, 1, 2}; double sign = 1; };

struct TypeBuild {
  Recipe R;
  BlockType bt;
  // (y0 + 12 y1 + 144 y2) -> cell (or -1 when identically zero), sign
  std::vector<int> cell_of;
  std::vector<signed char> sign_of;
};

void layout_type(TypeBuild& T) {
  BlockType& bt = T.bt;
  T.cell_of.assign(1728, -1);
  T.sign_of.assign(1728, 0);
  bt.cells.clear();
  if (bt.pack_sym == 0) {
    for (int y0 = 0; y0 < 12; ++y0)
      for (int y1 = 0; y1 < 12; ++y1)
        for (int y2 = 0; y2 < 12; ++y2) {
          int key = y0 + 12 * y1 + 144 * y2;
          T.cell_of[key] = (int)bt.cells.size();
          T.sign_of[key] = 1;
          bt.cells.push_back(key);
        }
  } else {
    int p = bt.pack_p, q = bt.pack_q, r = bt.pack_r;
    for (int a = 0; a < 12; ++a)
      for (int b = (bt.pack_sym > 0 ? a : a + 1); b < 12; ++b)
        for (int c = 0; c < 12; ++c) {
          int y[3];
          y[p] = a; y[q] = b; y[r] = c;
          int key = y[0] + 12 * y[1] + 144 * y[2];
          int cell = (int)bt.cells.size();
          bt.cells.push_back(key);
          T.cell_of[key] = cell;
          T.sign_of[key] = 1;
          if (a != b) {  // the mirrored pair
            int z[3];
            z[p] = b; z[q] = a; z[r] = c;
            int k2 = z[0] + 12 * z[1] + 144 * z[2];
            T.cell_of[k2] = cell;
            T.sign_of[k2] = (signed char)bt.pack_sym;
          }
        }
  }
  bt.ncell = (int)bt.cells.size();
}

}  // namespace

const char* field_name(int f) {
  static const char* names[NFIELDS] = {"p", "n", "Sigma+", "Sigma0", "Sigma-", "Xi0",
                                       "Xi-", "Lambda", "Xu", "Xd", "Xs"};
  return (f >= 0 && f < NFIELDS) ? names[f] : "?";
}

// Eqs. (2.2), (2.3): eps_abc (q1_a C gamma5 q2_b) q3_c with coefficients
const std::vector<Mono>& field_monomials(int f) {
  static const std::vector<std::vector<Mono>> table = {
      /* p      */ {{+1.0, {FU, FD, FU}}},
      /* n      */ {{-1.0, {FU, FD, FD}}},
      /* Sigma+ */ {{-1.0, {FU, FS, FU}}},
      /* Sigma0 */ {{kR2, {FD, FS, FU}}, {-kR2, {FS, FU, FD}}},
      /* Sigma- */ {{-1.0, {FD, FS, FD}}},
      /* Xi0    */ {{+1.0, {FU, FS, FS}}},
      /* Xi-    */ {{-1.0, {FD, FS, FS}}},
      /* Lambda */ {{kR6, {FD, FS, FU}}, {kR6, {FS, FU, FD}}, {-2.0 * kR6, {FU, FD, FS}}},
      /* Xu     */ {{1.0, {FD, FS, FU}}},
      /* Xd     */ {{1.0, {FS, FU, FD}}},
      /* Xs     */ {{1.0, {FU, FD, FS}}},
  };
  return table[f];
}

// Octet-octet channel list, reconstructed from the paper's "52 channels from
// NN to Xi Xi" (Sec. 1, Sec. 4 (iii)): in each strangeness sector the
// particle-basis sink pairs of minimal |I3| (zero total charge, +1 for
// S = -1), with every sink pair of the sector as a source (1+9+36+9+1 = 56),
// minus the four channels that vanish identically for u = d: a channel that
// is its own image under u <-> d with an odd sign (Lambda -> -Lambda,
// Sigma0 -> Sigma0), i.e. LL|LS0, LS0|LL, LS0|S0S0, S0S0|LS0.  52 remain.
const std::vector<ChannelDef>& channel_table() {
  static const std::vector<ChannelDef> table = [] {
    const std::vector<std::vector<std::pair<int, int>>> sectors = {
        {{P, N}},
        {{P, LAM}, {P, SIG0}, {N, SIGP}},
        {{P, XIM}, {N, XI0}, {LAM, LAM}, {LAM, SIG0}, {SIGP, SIGM}, {SIG0, SIG0}},
        {{LAM, XI0}, {SIGP, XIM}, {SIG0, XI0}},
        {{XI0, XIM}},
    };
    // u <-> d image of each field and its sign (Eqs. (2.2)-(2.3))
    const int img[NFIELDS] = {N, P, SIGM, SIG0, SIGP, XIM, XI0, LAM, XD, XU, XS};
    const int sgn[NFIELDS] = {1, 1, 1, 1, 1, -1, -1, -1, -1, -1, -1};
    std::vector<ChannelDef> t;
    for (auto& sec : sectors)
      for (auto& snk : sec)
        for (auto& src : sec) {
          ChannelDef c{{snk.first, snk.second, src.first, src.second}};
          bool self = true;
          int sign = 1;
          for (int b = 0; b < 4; ++b) {
            self = self && img[c.b[b]] == c.b[b];
            sign *= sgn[c.b[b]];
          }
          if (self && sign < 0) continue;  // identically zero in the isospin limit
          t.push_back(c);
        }
    return t;
  }();
  return table;
}

namespace {

// Reorder one term's compressed gather lists (entries [xi][i][held], side 1
// and side 2) for the shared-memory banks of the quad-lane kernels.  There a
// half-warp gathers, for one entry slot (i, held), the cells of four
// consecutive shared indices, each a 32-byte run (four spins) of the slab: the
// four cells take one pass of the banks when their cell indices differ mod 4
// (or coincide), else one pass per cell of the most used residue.  Any order
// of the shared indices (the same on both sides, they are paired) and of the
// entries of each sum gives the same product, and a zero-coefficient entry
// may name any cell: so, greedily, each group of four indices is filled with
// the candidate (among the next 48 unused) that adds the fewest passes, its
// entries put into the slots where they add the fewest, and its zero entries
// pointed at a cell the slot already reads.
void order_for_banks(int K, int n1, int nh1, int n2, int nh2, std::vector<unsigned short>& e1,
                     std::vector<unsigned short>& e2) {
  const int n[2] = {n1, n2}, nh[2] = {nh1, nh2}, r1 = n1 * nh1, r2 = n2 * nh2;
  if (K < 2 || (int)e1.size() != K * r1 || (int)e2.size() != K * r2) return;
  std::vector<unsigned short>* src[2] = {&e1, &e2};
  std::vector<unsigned short> out[2] = {std::vector<unsigned short>(e1.size()), std::vector<unsigned short>(e2.size())};
  struct Slot { int cell[4]; int nc; };
  std::vector<Slot> st(r1 + r2);
  auto slot_of = [&](int side, int i, int h) { return side == 0 ? i * nh1 + h : r1 + i * nh2 + h; };
  auto increase = [&](const Slot& s, int c) {
    int cnt[4] = {0, 0, 0, 0}, mx = 0;
    for (int j = 0; j < s.nc; ++j) {
      if (s.cell[j] == c) return 0;
      mx = std::max(mx, ++cnt[s.cell[j] & 3]);
    }
    return std::max(mx, cnt[c & 3] + 1) - mx;
  };
  auto add = [&](Slot& s, int c) {
    for (int j = 0; j < s.nc; ++j)
      if (s.cell[j] == c) return;
    if (s.nc < 4) s.cell[s.nc++] = c;
  };
  // cost of index k in the current group; with pos >= 0 also write it there
  auto place = [&](int k, int pos) {
    int tot = 0;
    for (int side = 0; side < 2; ++side) {
      const int nn = n[side], hh = nh[side];
      for (int h = 0; h < hh; ++h) {
        int slot_used[64] = {0};
        int assign[64];
        for (int pass = 0; pass < 2; ++pass)  // real entries first, then zeros
          for (int i = 0; i < nn; ++i) {
            const unsigned short e = (*src[side])[(k * nn + i) * hh + h];
            const bool zero = (e >> 11) == 31;
            if (zero != (pass == 1)) continue;
            int best = -1, best_inc = 1 << 30;
            for (int sl = 0; sl < nn; ++sl) {
              if (slot_used[sl]) continue;
              const int inc = zero ? 0 : increase(st[slot_of(side, sl, h)], e & 1023);
              if (inc < best_inc) { best_inc = inc; best = sl; }
            }
            slot_used[best] = 1;
            assign[i] = best;
            tot += best_inc;
          }
        if (pos < 0) continue;
        for (int i = 0; i < nn; ++i) {
          unsigned short e = (*src[side])[(k * nn + i) * hh + h];
          Slot& s = st[slot_of(side, assign[i], h)];
          if ((e >> 11) == 31 && s.nc > 0) e = (unsigned short)((e & ~1023u) | (unsigned)s.cell[0]);
          add(s, e & 1023);
          out[side][(pos * nn + assign[i]) * hh + h] = e;
        }
      }
    }
    return tot;
  };
  if (n1 > 64 || n2 > 64) return;
  std::vector<char> used(K, 0);
  int seed = 0, pos = 0;
  while (pos < K) {
    for (Slot& s : st) s.nc = 0;
    while (used[seed]) ++seed;
    place(seed, pos++);
    used[seed] = 1;
    for (int gi = 1; gi < 4 && pos < K; ++gi) {
      int best = -1, best_cost = 1 << 30;
      for (int k = seed, seen = 0; k < K && seen < 48; ++k) {
        if (used[k]) continue;
        ++seen;
        const int c = place(k, -1);
        if (c < best_cost) { best_cost = c; best = k; }
      }
      place(best, pos++);
      used[best] = 1;
    }
  }
  e1.swap(out[0]);
  e2.swap(out[1]);
}

// Split every slab group into chunks of whole channels whose compressed
// tables fit NBS_CHUNK_ENTRIES, and balance each chunk's items over warps.
// Measured cost of one 8-index step of the quad-lane contraction per run
// form (SM cycles of one of 16 warps, fitted to per-warp timings of the
// 52-channel tables at 16^3; shapes 0 and 2 run as their mirrors 3 and 1),
// of starting a run, and of a channel flush.
double quad_step_cost(int form, int ent) {
  switch (form) {
    case 5: return 799;
    case 7: return 1035;
    default: return 926 + 43.0 * ent;  // run-time lengths
  }
}
constexpr double QUAD_RUN_COST = 671, QUAD_FLUSH_COST = 893;

int quad_form(const TermHdr& th) {
  if ((th.shape == 0 && th.n1 == 8 && th.n2 == 2) || (th.shape == 1 && th.n1 == 2 && th.n2 == 2) ||
      (th.shape == 2 && th.n1 == 2 && th.n2 == 2) || (th.shape == 3 && th.n1 == 2 && th.n2 == 8))
    return th.shape + 4;
  return th.shape;
}

// Split every slab group into chunks of whole channels whose compressed
// tables fit NBS_CHUNK_ENTRIES, and balance each chunk's work over warps.
void build_chunks(Plan& plan) {
  plan.chunks.clear();
  plan.chunk_tab.clear();
  plan.chunk_items.clear();
  plan.quad_chunks.clear();
  plan.quad_segs.clear();
  plan.max_quad_segs = 0;
  plan.term_tab_off.assign(2 * plan.terms.size(), 0);
  plan.coef_codes.clear();
  plan.chunks_ok = false;
  auto code_of = [&](double c) -> int {
    const double a = std::fabs(c);
    for (size_t i = 0; i < plan.coef_codes.size(); ++i)
      if (std::fabs(plan.coef_codes[i] - a) <= 1e-12 * std::max(1.0, a)) return (int)i;
    plan.coef_codes.push_back(a);
    return (int)plan.coef_codes.size() - 1;
  };
  auto held = [](const TermHdr& th, int& nh1, int& nh2) {
    nh1 = 1 << ((th.shape & 1) + (th.shape >> 1 & 1));
    nh2 = 4 / nh1;
  };
  auto term_entries = [&](const TermHdr& th) {
    int nh1, nh2;
    held(th, nh1, nh2);
    auto pad8 = [](int n) { return (n + 7) / 8 * 8; };
    return pad8(th.K * nh1 * th.n1) + pad8(th.K * nh2 * th.n2);
  };
  // one table run: a channel's terms of one fixed form (lists of whole 16-byte
  // rows), or a single term
  struct Run { int form, n1, n2, nh1, nh2, K, local, t1, t2, swap; };
  for (const GroupHdr& g : plan.groups) {
    if (g.ncell1 > 1024 || g.ncell2 > 1024) return;
    int c = 0;
    while (c < g.nch) {
      // take whole channels while the table fits
      int c_end = c, len = 0;
      while (c_end < g.nch) {
        const int ci = plan.group_ch[g.ch_off + c_end];
        int n = 0;
        for (int t = plan.ch_term_begin[ci]; t < plan.ch_term_begin[ci + 1]; ++t) n += term_entries(plan.terms[t]);
        if (len + n > NBS_CHUNK_ENTRIES) break;
        len += n;
        ++c_end;
      }
      if (c_end == c) return;  // one channel alone exceeds a chunk
      ChunkHdr ck = {};
      ck.base1 = g.base1; ck.ncell1 = g.ncell1; ck.base2 = g.base2; ck.ncell2 = g.ncell2;
      ck.ch_off = g.ch_off + c;
      ck.nch = c_end - c;
      ck.ch_local0 = c;
      ck.tab_off = (int)plan.chunk_tab.size();
      ck.item_off = (int)plan.chunk_items.size() / 2;
      std::vector<std::pair<int, int>> its;
      std::vector<double> cost;
      std::vector<Run> runs;
      for (int local = c; local < c_end; ++local) {
        const int ci = plan.group_ch[g.ch_off + local];
        // the channel's runs: terms of one fixed form whose lists are whole
        // 16-byte rows go together, in order of first appearance
        std::vector<std::vector<int>> members;
        std::vector<int> run_form;
        for (int t = plan.ch_term_begin[ci]; t < plan.ch_term_begin[ci + 1]; ++t) {
          const TermHdr& th = plan.terms[t];
          int nh1, nh2;
          held(th, nh1, nh2);
          const int form = quad_form(th);
          const bool whole = (th.K * nh1 * th.n1) % 8 == 0 && (th.K * nh2 * th.n2) % 8 == 0;
          int r = -1;
          if (form >= 4 && whole)
            for (size_t j = 0; j < members.size(); ++j)
              if (run_form[j] == form) r = (int)j;
          if (r < 0) {
            members.emplace_back();
            run_form.push_back(form >= 4 && whole ? form : -1);
            r = (int)members.size() - 1;
          }
          members[r].push_back(t);
        }
        // shapes 0 and 2 run as shapes 3 and 1 with the two sides exchanged
        // (the product then lands transposed in alpha1, alpha2): a channel's
        // runs with exchanged sides go last, so a warp flushes at most twice
        std::stable_sort(members.begin(), members.end(), [&](const std::vector<int>& x, const std::vector<int>& y) {
          return (plan.terms[x[0]].shape % 2 == 0) < (plan.terms[y[0]].shape % 2 == 0);
        });
        for (const std::vector<int>& mem : members) {
          const TermHdr& t0 = plan.terms[mem[0]];
          Run run;
          run.form = quad_form(t0);
          run.n1 = t0.n1;
          run.n2 = t0.n2;
          held(t0, run.nh1, run.nh2);
          run.K = 0;
          run.local = t0.pad - c;
          run.swap = t0.shape % 2 == 0;
          std::vector<unsigned short> ents[2];
          std::vector<int> koff;
          for (int t : mem) {
            const TermHdr& th = plan.terms[t];
            koff.push_back(run.K);
            run.K += th.K;
            for (int side = 0; side < 2; ++side) {
              const int n = side == 0 ? th.K * run.nh1 * th.n1 : th.K * run.nh2 * th.n2;
              const int off = side == 0 ? th.off1 : th.off2;
              const int base = side == 0 ? g.base1 : g.base2;
              const auto& cells = side == 0 ? plan.ent1_cell : plan.ent2_cell;
              const auto& coefs = side == 0 ? plan.ent1_coef : plan.ent2_coef;
              for (int i = 0; i < n; ++i) {
                const int cell = cells[off + i] - base;
                const double cf = coefs[off + i];
                if (cell < 0 || cell >= 1024) return;
                int code = 31;  // code 31: zero coefficient (padding)
                if (cf != 0.0) {
                  code = code_of(cf);
                  if (code >= 31) return;
                }
                ents[side].push_back((unsigned short)(cell | ((cf < 0) << 10) | (code << 11)));
              }
            }
          }
          // the members of a run share channel and form: any of the run's
          // shared indices may stand at any member's position
          order_for_banks(run.K, run.n1, run.nh1, run.n2, run.nh2, ents[0], ents[1]);
          const int r1 = run.nh1 * run.n1, r2 = run.nh2 * run.n2;
          run.t1 = (int)plan.chunk_tab.size() - ck.tab_off;
          plan.chunk_tab.insert(plan.chunk_tab.end(), ents[0].begin(), ents[0].end());
          while ((plan.chunk_tab.size() - ck.tab_off) % 8) plan.chunk_tab.push_back((unsigned short)(0x1F << 11));
          run.t2 = (int)plan.chunk_tab.size() - ck.tab_off;
          plan.chunk_tab.insert(plan.chunk_tab.end(), ents[1].begin(), ents[1].end());
          while ((plan.chunk_tab.size() - ck.tab_off) % 8) plan.chunk_tab.push_back((unsigned short)(0x1F << 11));
          for (size_t j = 0; j < mem.size(); ++j) {
            const int t = mem[j];
            const TermHdr& th = plan.terms[t];
            plan.term_tab_off[2 * t] = run.t1 + koff[j] * r1;
            plan.term_tab_off[2 * t + 1] = run.t2 + koff[j] * r2;
            for (int k0 = 0; k0 < th.K; k0 += 32) {
              // warp instructions per step of the pair-lane kernels ~ a fixed part
              // plus one part per gather entry of a shared index
              const int nkb = (std::min(32, th.K - k0) + 15) / 16;  // 16 indices per step
              its.push_back({t, k0});
              cost.push_back(nkb * (26.0 + r1 + r2));
            }
          }
          runs.push_back(run);
        }
      }
      ck.tab_len = (int)plan.chunk_tab.size() - ck.tab_off;
      // contiguous per-warp item ranges of about equal cost, and the partial-sum
      // slots each warp needs (one per channel its range touches)
      {
        double total = 0;
        for (double x : cost) total += x;
        int w = 0;
        double acc = 0;
        ck.warp_off[0] = 0;
        for (size_t i = 0; i < its.size(); ++i) {
          acc += cost[i];
          if (w < NBS_CHUNK_WARPS - 1 && acc >= total * (w + 1) / NBS_CHUNK_WARPS) ck.warp_off[++w] = (int)i + 1;
        }
        while (w < NBS_CHUNK_WARPS) ck.warp_off[++w] = (int)its.size();
        ck.out_base[0] = 0;
        for (int ww = 0; ww < NBS_CHUNK_WARPS; ++ww) {
          int n = 0;
          ck.cfirst[ww] = 0;
          if (ck.warp_off[ww + 1] > ck.warp_off[ww]) {
            const int c0 = plan.terms[its[ck.warp_off[ww]].first].pad - c;
            const int c1 = plan.terms[its[ck.warp_off[ww + 1] - 1].first].pad - c;
            ck.cfirst[ww] = c0;
            n = c1 - c0 + 1;
          }
          ck.out_base[ww + 1] = ck.out_base[ww] + n;
        }
        ck.nslot = ck.out_base[NBS_CHUNK_WARPS];
      }
      QuadChunkHdr qk = {};
      qk.base1 = ck.base1; qk.ncell1 = ck.ncell1; qk.base2 = ck.base2; qk.ncell2 = ck.ncell2;
      qk.ch_off = ck.ch_off; qk.nch = ck.nch; qk.tab_off = ck.tab_off; qk.tab_len = ck.tab_len;
      qk.ch_local0 = ck.ch_local0;
      {
        // the runs' 8-index steps in order, each with its measured cost; a warp's
        // range also pays one run start per run and one flush per channel it
        // touches.  Cut into NBS_QUAD_WARPS contiguous ranges whose largest
        // cost is smallest (bisection on that cost, greedy fill).
        std::vector<int> srun, sk;
        std::vector<double> scost;
        for (size_t r = 0; r < runs.size(); ++r) {
          const Run& run = runs[r];
          const double sc = quad_step_cost(run.swap ? (run.form ^ 3) : run.form, run.nh1 * run.n1 + run.nh2 * run.n2);
          for (int k = 0; k < run.K; k += 8) {
            srun.push_back((int)r);
            sk.push_back(k);
            scost.push_back(sc);
          }
        }
        const int nsteps = (int)scost.size();
        auto add_cost = [&](int s, bool first) {  // cost of step s appended to a range
          double x = scost[s];
          if (first || srun[s] != srun[s - 1]) x += QUAD_RUN_COST;
          if (first || runs[srun[s]].local != runs[srun[s - 1]].local || runs[srun[s]].swap != runs[srun[s - 1]].swap)
            x += QUAD_FLUSH_COST;
          return x;
        };
        auto fill = [&](double cap, std::vector<int>* cut) {  // warps used by a greedy fill
          int w = 0;
          double acc = 0;
          if (cut) (*cut)[0] = 0;
          for (int s = 0; s < nsteps; ++s) {
            const bool first = s == 0 || (cut && (*cut)[w] == s);
            double x = add_cost(s, first);
            if (!first && acc + x > cap) {
              ++w;
              if (w >= NBS_QUAD_WARPS) return w + 1;
              if (cut) (*cut)[w] = s;
              x = add_cost(s, true);
              acc = 0;
            }
            acc += x;
          }
          if (cut)
            for (int ww = w + 1; ww <= NBS_QUAD_WARPS; ++ww) (*cut)[ww] = nsteps;
          return w + 1;
        };
        double lo = 0, hi = 0;
        for (int s = 0; s < nsteps; ++s) {
          hi += add_cost(s, true);
          lo = std::max(lo, add_cost(s, true));
        }
        for (int it = 0; it < 60 && hi - lo > 1e-6 * hi; ++it) {
          const double mid = 0.5 * (lo + hi);
          if (fill(mid, nullptr) <= NBS_QUAD_WARPS) hi = mid;
          else lo = mid;
        }
        std::vector<int> cut(NBS_QUAD_WARPS + 1, nsteps);
        fill(hi, &cut);
        const int seg0 = (int)plan.quad_segs.size();
        qk.out_base[0] = 0;
        for (int ww = 0; ww < NBS_QUAD_WARPS; ++ww) {
          qk.seg_base[ww] = (int)plan.quad_segs.size();
          int n = 0;
          qk.cfirst[ww] = 0;
          if (cut[ww + 1] > cut[ww]) {
            const int c0 = runs[srun[cut[ww]]].local, c1 = runs[srun[cut[ww + 1] - 1]].local;
            qk.cfirst[ww] = c0;
            n = c1 - c0 + 1;
          }
          qk.out_base[ww + 1] = qk.out_base[ww] + n;
          for (int s = cut[ww]; s < cut[ww + 1]; ++s) {
            const Run& run = runs[srun[s]];
            const int kend = std::min(run.K, sk[s] + 8);
            if (s > cut[ww] && srun[s - 1] == srun[s]) {
              plan.quad_segs.back().kend = kend;
              continue;
            }
            QuadSeg sg;
            sg.form = run.swap ? (run.form ^ 3) | 8 : run.form;  // 0 <-> 3, 2 <-> 1, 4 <-> 7, 6 <-> 5
            sg.t1 = run.swap ? run.t2 : run.t1;
            sg.t2 = run.swap ? run.t1 : run.t2;
            sg.kbeg = sk[s];
            sg.kend = kend;
            sg.local = run.local;
            sg.n1 = run.swap ? run.n2 : run.n1;
            sg.n2 = run.swap ? run.n1 : run.n2;
            plan.quad_segs.push_back(sg);
          }
        }
        qk.seg_base[NBS_QUAD_WARPS] = (int)plan.quad_segs.size();
        qk.nslot = qk.out_base[NBS_QUAD_WARPS];
        plan.max_quad_segs = std::max(plan.max_quad_segs, (int)plan.quad_segs.size() - seg0);
      }
      plan.quad_chunks.push_back(qk);
      for (auto& it : its) {
        plan.chunk_items.push_back(it.first);
        plan.chunk_items.push_back(it.second);
      }
      plan.chunks.push_back(ck);
      c = c_end;
    }
  }
  // code 31 is reserved for zero coefficients
  if (plan.coef_codes.size() > 31) return;
  plan.chunks_ok = true;
}

}  // namespace

std::string compile_plan(const std::vector<int>& ids, Plan& plan, int nflav) {
  plan = Plan();
  if (nflav != 2 && nflav != 3) return "flavours must be 2 (u = d, s) or 3 (u, d, s)";
  plan.nflav = nflav;
  const auto& table = channel_table();
  // id = channel + n * block: block o3 + 2 o4 selects the source spins
  // alpha3 in {2 o3, 2 o3 + 1}, alpha4 in {2 o4, 2 o4 + 1} (block 0: the upper components)
  const int nbase = (int)table.size();
  for (int id : ids) {
    if (id < 0 || id >= NBS_SPIN_BLOCKS * nbase) {
      std::ostringstream os;
      os << "channel id " << id << " outside [0, " << NBS_SPIN_BLOCKS * nbase << ")";
      return os.str();
    }
  }
  plan.channels = ids;

  // ---- stored block types over the sink fields in use -----------------------
  bool used[NFIELDS] = {};
  for (int id : ids) { used[table[id % nbase].b[0]] = used[table[id % nbase].b[1]] = true; }
  std::vector<TypeBuild> types;
  FieldMap fmap[NFIELDS];
  for (int f = 0; f < NFIELDS; ++f) {
    if (!used[f]) continue;
    Recipe R;
    if (!field_recipe(f, R, nflav)) return std::string("field ") + field_name(f) + " has no block pattern";
    bool found = false;
    for (int t = 0; t < (int)types.size() && !found; ++t) {
      for (auto& pi : kPerm3) {
        Recipe C = compose(types[t].R, pi, nflav);
        for (double s : {1.0, -1.0}) {
          if (equal_scaled(R, C, s)) {
            fmap[f].type = t;
            std::copy(pi, pi + 3, fmap[f].pi);
            fmap[f].sign = s;
            found = true;
            break;
          }
        }
        if (found) break;
      }
    }
    if (found) continue;
    TypeBuild T;
    T.R = R;
    const int pairs[3][3] = {{0, 1, 2}, {1, 2, 0}, {0, 2, 1}};
    for (auto& pr : pairs) {
      int sw[3] = {0, 1, 2};
      std::swap(sw[pr[0]], sw[pr[1]]);
      Recipe C = compose(R, sw, nflav);
      int sym = equal_scaled(C, R, 1.0) ? 1 : (equal_scaled(C, R, -1.0) ? -1 : 0);
      if (sym) {
        T.bt.pack_p = pr[0]; T.bt.pack_q = pr[1]; T.bt.pack_r = pr[2]; T.bt.pack_sym = sym;
        break;
      }
    }
    for (auto& kv : R) T.bt.terms.push_back({kv.first[0], {kv.first[1], kv.first[2], kv.first[3]}, kv.second});
    layout_type(T);
    fmap[f].type = (int)types.size();
    types.push_back(std::move(T));
  }
  int off = 0;
  for (auto& T : types) { T.bt.cell_off = off; off += T.bt.ncell; }
  plan.ncells = off;

  // ---- contraction terms -----------------------------------------------------
  plan.ch_term_begin.push_back(0);
  for (int ci = 0; ci < (int)ids.size(); ++ci) {
    const ChannelDef& ch = table[ids[ci] % nbase];
    const int sblock = ids[ci] / nbase;
    const int soff[2] = {sblock & 1, sblock >> 1};  // source spin pair offsets of alpha3, alpha4
    const int B1 = ch.b[0], B2 = ch.b[1];
    int cf1[3], cf2[3];
    canonical_flavours(B1, cf1);
    canonical_flavours(B2, cf2);
    {
      int nl = 0, fl[3] = {0, 0, 0};
      for (int k = 0; k < 3; ++k) {
        nl += (cf1[k] != FS) + (cf2[k] != FS);
        ++fl[lflav(cf1[k], nflav)];
        ++fl[lflav(cf2[k], nflav)];
      }
      plan.ch_nl.push_back(nl);
      plan.ch_fl.insert(plan.ch_fl.end(), fl, fl + 3);
    }
    for (const Mono& m3 : field_monomials(ch.b[2])) {
      for (const Mono& m4 : field_monomials(ch.b[3])) {
        int src[6] = {m3.q[0], m3.q[1], m3.q[2], m4.q[0], m4.q[1], m4.q[2]};
        const double c34 = m3.c * m4.c;
        for (int mask = 0; mask < 64; ++mask) {
          if (__builtin_popcount(mask) != 3) continue;
          int S[3], Sc[3], ns = 0, nc = 0;
          for (int k = 0; k < 6; ++k) {
            if (mask >> k & 1) S[ns++] = k; else Sc[nc++] = k;
          }
          // flavour content of S must be B1's, of the complement B2's
          int fs[3] = {src[S[0]], src[S[1]], src[S[2]]}, fc[3] = {src[Sc[0]], src[Sc[1]], src[Sc[2]]};
          std::sort(fs, fs + 3);
          std::sort(fc, fc + 3);
          if (!std::equal(fs, fs + 3, cf1) || !std::equal(fc, fc + 3, cf2)) continue;
          int P0[6] = {S[0], S[1], S[2], Sc[0], Sc[1], Sc[2]};
          const int sign0 = perm_sign(P0, 6);
          bool on1[6];
          for (int k = 0; k < 6; ++k) on1[k] = mask >> k & 1;
          // side of each source baryon's eps / Cg5 (majority) and projector (its third slot)
          int fside[2], pside[2];
          for (int b = 0; b < 2; ++b) {
            int cnt = on1[3 * b] + on1[3 * b + 1] + on1[3 * b + 2];
            fside[b] = cnt >= 2 ? 1 : 2;
            pside[b] = on1[3 * b + 2] ? 1 : 2;
          }
          // shared indices: (kind 0 = colour / 1 = spin, slot), canonical order
          std::vector<std::pair<int, int>> xi;
          for (int b = 0; b < 2; ++b) {
            for (int k = 3 * b; k < 3 * b + 3; ++k)
              if ((on1[k] ? 1 : 2) != fside[b]) xi.push_back({0, k});
            for (int k = 3 * b; k < 3 * b + 2; ++k)
              if ((on1[k] ? 1 : 2) != fside[b]) xi.push_back({1, k});
          }
          std::sort(xi.begin(), xi.end());
          int K = 1;
          for (auto& x : xi) K *= x.first == 0 ? 3 : 4;
          const int shape = (pside[0] == 1 ? 1 : 0) | (pside[1] == 1 ? 2 : 0);

          std::vector<int> cells_side[2];
          std::vector<double> coef_side[2];
          int nmax[2] = {0, 0};
          for (int side = 1; side <= 2; ++side) {
            const int field = side == 1 ? B1 : B2;
            const int* cf = side == 1 ? cf1 : cf2;
            const int* slots = side == 1 ? S : Sc;
            // rho: canonical position -> index into slots (flavour preserving)
            int rho[3];
            bool taken[3] = {};
            for (int p = 0; p < 3; ++p) {
              rho[p] = -1;
              for (int i = 0; i < 3; ++i)
                if (!taken[i] && src[slots[i]] == cf[p]) { rho[p] = i; taken[i] = true; break; }
              if (rho[p] < 0) return "internal: no flavour-preserving map";
            }
            const double side_coef = perm_sign(rho, 3) * (side == 1 ? sign0 * c34 : 1.0);
            const FieldMap& fm = fmap[field];
            const TypeBuild& T = types[fm.type];
            int nheld = (pside[0] == side) + (pside[1] == side);
            std::vector<std::vector<std::pair<int, double>>> lists;
            for (int k = 0; k < K; ++k) {
              int col[6], spin[6];
              std::fill(col, col + 6, -1);
              std::fill(spin, spin + 6, -1);
              int rem = k;
              for (int i = (int)xi.size() - 1; i >= 0; --i) {
                int base = xi[i].first == 0 ? 3 : 4;
                int v = rem % base;
                rem /= base;
                (xi[i].first == 0 ? col : spin)[xi[i].second] = v;
              }
              for (int h = 0; h < (1 << nheld); ++h) {
                int sp[6];
                std::copy(spin, spin + 6, sp);
                int bit = 0;
                for (int b = 0; b < 2; ++b) {
                  if (pside[b] != side) continue;
                  sp[3 * b + 2] = 2 * soff[b] + ((h >> bit) & 1);  // projector: third slot's spin = alpha_{3/4}
                  ++bit;
                }
                // free indices of this side's slots
                int fcol[3], nfc = 0, fsp[3], nfs = 0;
                for (int i = 0; i < 3; ++i) {
                  if (col[slots[i]] < 0) fcol[nfc++] = slots[i];
                  if (sp[slots[i]] < 0) fsp[nfs++] = slots[i];
                }
                std::map<int, double> acc;
                int ncc = 1, nsc = 1;
                for (int i = 0; i < nfc; ++i) ncc *= 3;
                for (int i = 0; i < nfs; ++i) nsc *= 4;
                for (int cc = 0; cc < ncc; ++cc) {
                  int c6[6];
                  std::copy(col, col + 6, c6);
                  for (int i = 0, r = cc; i < nfc; ++i, r /= 3) c6[fcol[i]] = r % 3;
                  double ce = 1;
                  for (int b = 0; b < 2; ++b)
                    if (fside[b] == side) ce *= eps3(c6[3 * b], c6[3 * b + 1], c6[3 * b + 2]);
                  if (ce == 0) continue;
                  for (int ss = 0; ss < nsc; ++ss) {
                    int s6[6];
                    std::copy(sp, sp + 6, s6);
                    for (int i = 0, r = ss; i < nfs; ++i, r /= 4) s6[fsp[i]] = r % 4;
                    double cs = 1;
                    for (int b = 0; b < 2; ++b)
                      if (fside[b] == side) cs *= kCG5[s6[3 * b]][s6[3 * b + 1]];
                    if (cs == 0) continue;
                    // field-block arguments in canonical order
                    int y[3];
                    for (int p = 0; p < 3; ++p) {
                      int sl = slots[rho[p]];
                      y[p] = 3 * s6[sl] + c6[sl];
                    }
                    // FB^field(y) = sign * FB^T(y_pi0, y_pi1, y_pi2)
                    int yt[3] = {y[fm.pi[0]], y[fm.pi[1]], y[fm.pi[2]]};
                    int key = yt[0] + 12 * yt[1] + 144 * yt[2];
                    int cell = T.cell_of[key];
                    if (cell < 0) continue;
                    double c = ce * cs * fm.sign * T.sign_of[key] * side_coef;
                    acc[T.bt.cell_off + cell] += c;
                  }
                }
                std::vector<std::pair<int, double>> lst;
                for (auto& kv : acc)
                  if (std::fabs(kv.second) > 1e-13) lst.push_back(kv);
                nmax[side - 1] = std::max(nmax[side - 1], (int)lst.size());
                lists.push_back(std::move(lst));
              }
            }
            // entries of step k ordered [i][h], i padded to an even count with zero coefficients
            nmax[side - 1] += nmax[side - 1] & 1;
            const int nh = 1 << nheld;
            for (int k = 0; k < K; ++k)
              for (int i = 0; i < nmax[side - 1]; ++i)
                for (int hh = 0; hh < nh; ++hh) {
                  const auto& lst = lists[k * nh + hh];
                  if (i < (int)lst.size()) {
                    cells_side[side - 1].push_back(lst[i].first);
                    coef_side[side - 1].push_back(lst[i].second);
                  } else {
                    // padding: zero coefficient on a cell of the same stored type
                    cells_side[side - 1].push_back(T.bt.cell_off);
                    coef_side[side - 1].push_back(0.0);
                  }
                }
          }
          if (nmax[0] == 0 || nmax[1] == 0) continue;  // identically zero term
          TermHdr th;
          th.ch = ci;
          th.K = K;
          th.shape = shape;
          th.n1 = nmax[0];
          th.n2 = nmax[1];
          th.off1 = (int)plan.ent1_cell.size();
          th.off2 = (int)plan.ent2_cell.size();
          th.pad = 0;
          plan.ent1_cell.insert(plan.ent1_cell.end(), cells_side[0].begin(), cells_side[0].end());
          plan.ent1_coef.insert(plan.ent1_coef.end(), coef_side[0].begin(), coef_side[0].end());
          plan.ent2_cell.insert(plan.ent2_cell.end(), cells_side[1].begin(), cells_side[1].end());
          plan.ent2_coef.insert(plan.ent2_coef.end(), coef_side[1].begin(), coef_side[1].end());
          plan.terms.push_back(th);
          const int nh1 = 1 << ((shape & 1) + (shape >> 1 & 1));
          const int nh2 = 4 / nh1;
          plan.cmac_per_q += 64.0 * K;
          plan.gathers_per_q += 4.0 * K * (nh1 * th.n1 + nh2 * th.n2);
        }
      }
    }
    plan.ch_term_begin.push_back((int)plan.terms.size());
  }
  // ---- keep only the stored cells some gather entry reads: the others would be built and transformed
  // for nothing.  Every type keeps its cells in their order, renumbered; the entries follow.
  {
    std::vector<char> used((size_t)plan.ncells, 0);
    for (int c : plan.ent1_cell) used[(size_t)c] = 1;
    for (int c : plan.ent2_cell) used[(size_t)c] = 1;
    std::vector<int> renum((size_t)plan.ncells, -1);
    int kept = 0;
    for (auto& T : types) {
      BlockType& bt = T.bt;
      std::vector<int> cells;
      for (int k = 0; k < bt.ncell; ++k)
        if (used[(size_t)(bt.cell_off + k)]) {
          renum[(size_t)(bt.cell_off + k)] = kept + (int)cells.size();
          cells.push_back(bt.cells[k]);
        }
      bt.cells = std::move(cells);
      bt.ncell = (int)bt.cells.size();
      bt.cell_off = kept;
      kept += bt.ncell;
    }
    for (int& c : plan.ent1_cell) c = renum[(size_t)c];
    for (int& c : plan.ent2_cell) c = renum[(size_t)c];
    plan.ncells = kept;
  }
  for (auto& T : types) plan.types.push_back(T.bt);

  // ---- slab groups for the momentum-slab contraction -------------------------
  {
    std::map<std::pair<int, int>, std::vector<int>> by_types;  // (type B1, type B2) -> channels
    for (int ci = 0; ci < (int)ids.size(); ++ci) {
      const ChannelDef& ch = table[ids[ci] % nbase];
      by_types[{fmap[ch.b[0]].type, fmap[ch.b[1]].type}].push_back(ci);
    }
    for (auto& kv : by_types) {
      GroupHdr g = {};
      const BlockType& t1 = types[kv.first.first].bt;
      const BlockType& t2 = types[kv.first.second].bt;
      g.base1 = t1.cell_off; g.ncell1 = t1.ncell;
      g.base2 = t2.cell_off; g.ncell2 = t2.ncell;
      g.ch_off = (int)plan.group_ch.size();
      g.nch = (int)kv.second.size();
      g.item_off = (int)plan.items.size() / 2;
      // items in channel order, with their cost (products plus gathers of 32 shared indices)
      std::vector<std::pair<int, int>> its;
      std::vector<double> cost;
      for (int local = 0; local < g.nch; ++local) {
        const int ci = kv.second[local];
        plan.group_ch.push_back(ci);
        for (int t = plan.ch_term_begin[ci]; t < plan.ch_term_begin[ci + 1]; ++t) {
          TermHdr& th = plan.terms[t];
          th.pad = local;
          const int nh1 = 1 << ((th.shape & 1) + (th.shape >> 1 & 1)), nh2 = 4 / nh1;
          for (int k0 = 0; k0 < th.K; k0 += 32) {
            its.push_back({t, k0});
            cost.push_back(64.0 + 4.0 * (nh1 * th.n1 + nh2 * th.n2));
          }
        }
      }
      double total = 0;
      for (double c : cost) total += c;
      // contiguous split into NBS_SLAB_WARPS ranges of about equal cost
      int w = 0;
      double acc = 0;
      g.warp_off[0] = 0;
      for (size_t i = 0; i < its.size(); ++i) {
        acc += cost[i];
        if (w < NBS_SLAB_WARPS - 1 && acc >= total * (w + 1) / NBS_SLAB_WARPS) g.warp_off[++w] = (int)i + 1;
      }
      while (w < NBS_SLAB_WARPS) g.warp_off[++w] = (int)its.size();
      // each warp's items span a contiguous range of group channels: one slot each
      g.out_base[0] = 0;
      for (int ww = 0; ww < NBS_SLAB_WARPS; ++ww) {
        int n = 0;
        g.cfirst[ww] = 0;
        if (g.warp_off[ww + 1] > g.warp_off[ww]) {
          const int c0 = plan.terms[its[g.warp_off[ww]].first].pad;
          const int c1 = plan.terms[its[g.warp_off[ww + 1] - 1].first].pad;
          g.cfirst[ww] = c0;
          n = c1 - c0 + 1;
        }
        g.out_base[ww + 1] = g.out_base[ww] + n;
      }
      g.nslot = g.out_base[NBS_SLAB_WARPS];
      for (auto& it : its) {
        plan.items.push_back(it.first);
        plan.items.push_back(it.second);
      }
      plan.groups.push_back(g);
    }
  }
  build_chunks(plan);
  build_row_chunks(plan, NBS_ROW_SMEM_LIMIT);
  return "";
}

}  // namespace nbs
