// plan_rows.cpp -- tables of the two-phase contraction (kernels_rows.cu).
//
// The gather lists of the effective blocks (Eq. (4.2); Sec. 4 (ii)) repeat
// heavily across terms and channels: over the 52 channels about 87 thousand
// (shared index, held spin) rows of each side are built from only a few
// thousand distinct sums of stored cells.  So, per chunk of channels of one
// slab group, every distinct row is listed once (phase A builds it per
// momentum for all four sink spins), and the product of Eq. (4.3) walks
// records that name, for each shared index xi~ and output source-spin pair s,
// the row of each side and a scale (phase B).
//
// A row is kept up to a scale: with m the smallest coefficient magnitude of
// its term side, its coefficients are m times +-1 or +-2, and it is stored
// with the sign that makes its first entry (lowest cell) positive.  The
// record's scale is then m1 m2 sign1 sign2, one of at most 31 values over a
// plan (a code into Plan::row_scales).
#include <algorithm>
#include <cmath>
#include <map>
#include <sstream>
#include <vector>

#include "plan.h"

namespace nbs {

namespace {

int held_count(int shape) { return 1 << ((shape & 1) + ((shape >> 1) & 1)); }

// held source spins (h1 of B1's list, h2 of B2's) feeding output pair s = alpha3 + 2 alpha4;
// shape bit 0: alpha3's projector on B1, bit 1: alpha4's projector on B1
void held_of(int shape, int s, int& h1, int& h2) {
  switch (shape) {
    case 0: h1 = 0; h2 = s; break;
    case 3: h1 = s; h2 = 0; break;
    case 1: h1 = s & 1; h2 = s >> 1; break;
    default: h1 = s >> 1; h2 = s & 1; break;
  }
}

using RowKey = std::vector<std::pair<int, int>>;  // (slab cell, integer coefficient), cells ascending

struct SideRows {
  std::map<RowKey, int> id;  // key -> provisional id
  std::vector<const RowKey*> keys;
  long long entries = 0;
  int add(const RowKey& k) {
    auto it = id.find(k);
    if (it != id.end()) return it->second;
    const int n = (int)keys.size();
    auto ins = id.emplace(k, n).first;
    keys.push_back(&ins->first);
    entries += (long long)k.size();
    return n;
  }
};

// one (xi~, held spin) row of a term side: canonical key, its sign, empty flag
struct RowOf {
  RowKey key;
  int sign = 1;
  bool empty = true;
};

struct TermRows {
  double m1 = 0, m2 = 0;
  std::vector<RowOf> r1, r2;  // [k * NH + h]
};

// rows of one term; false (with a reason) if a coefficient is not m * {+-1, +-2}
bool term_rows(const Plan& P, const TermHdr& th, int base1, int base2, TermRows& out, std::string& why) {
  const int nh1 = held_count(th.shape), nh2 = 4 / nh1;
  for (int side = 0; side < 2; ++side) {
    const int n = side ? th.n2 : th.n1, nh = side ? nh2 : nh1, off = side ? th.off2 : th.off1;
    const std::vector<int>& cells = side ? P.ent2_cell : P.ent1_cell;
    const std::vector<double>& coefs = side ? P.ent2_coef : P.ent1_coef;
    const int base = side ? base2 : base1, shift = side ? NBS_ROW_SLAB : 0;
    double m = 0;
    for (int i = 0; i < th.K * n * nh; ++i) {
      const double a = std::fabs(coefs[off + i]);
      if (a > 0 && (m == 0 || a < m)) m = a;
    }
    std::vector<RowOf>& rows = side ? out.r2 : out.r1;
    (side ? out.m2 : out.m1) = m;
    rows.assign((size_t)th.K * nh, RowOf());
    for (int k = 0; k < th.K; ++k)
      for (int h = 0; h < nh; ++h) {
        RowOf& r = rows[(size_t)k * nh + h];
        for (int i = 0; i < n; ++i) {
          const int e = off + (k * n + i) * nh + h;
          const double c = coefs[e];
          if (c == 0) continue;
          const double q = c / m;
          const int iq = (int)std::lround(q);
          if (std::fabs(q - iq) > 1e-9 || (std::abs(iq) != 1 && std::abs(iq) != 2)) {
            std::ostringstream os;
            os << "coefficient " << c << " is not +-1 or +-2 times " << m;
            why = os.str();
            return false;
          }
          const int cell = cells[e] - base;
          if (cell < 0 || cell >= NBS_ROW_SLAB) {
            why = "stored type larger than a slab side";
            return false;
          }
          r.key.push_back({cell + shift, iq});
        }
        if (r.key.empty()) continue;
        r.empty = false;
        std::sort(r.key.begin(), r.key.end());
        // merge equal cells (not expected: the compiler already sums them)
        RowKey mk;
        for (auto& e : r.key) {
          if (!mk.empty() && mk.back().first == e.first) mk.back().second += e.second;
          else mk.push_back(e);
        }
        mk.erase(std::remove_if(mk.begin(), mk.end(), [](const std::pair<int, int>& e) { return e.second == 0; }),
                 mk.end());
        if (mk.empty()) {
          r.key.clear();
          r.empty = true;
          continue;
        }
        for (auto& e : mk)
          if (std::abs(e.second) > 2) {
            why = "merged coefficient beyond +-2";
            return false;
          }
        r.sign = mk[0].second > 0 ? 1 : -1;
        if (r.sign < 0)
          for (auto& e : mk) e.second = -e.second;
        r.key = std::move(mk);
      }
  }
  return true;
}

int scale_code(std::vector<double>& scales, double v, std::string& why) {
  if (v == 0) return NBS_ROW_SCALES - 1;
  for (size_t i = 0; i < scales.size(); ++i)
    if (std::fabs(scales[i] - v) <= 1e-12 * std::fabs(v)) return (int)i;
  if ((int)scales.size() >= NBS_ROW_SCALES - 1) {
    why = "more than 31 distinct term scales";
    return -1;
  }
  scales.push_back(v);
  return (int)scales.size() - 1;
}

// contiguous split of the chunk's steps into NBS_ROW_WARPS ranges: a warp's
// cost is its steps plus kFlush per channel piece it holds; bisection on the
// largest cost, greedy fill
constexpr double kFlush = 2.0;

std::vector<int> split_steps(const std::vector<int>& step_ch) {
  const int n = (int)step_ch.size();
  auto fill = [&](double cap, std::vector<int>* starts) {
    int w = 0, cur = -1;
    double cost = 0;
    if (starts) starts->assign(1, 0);
    for (int i = 0; i < n; ++i) {
      double add = 1.0 + (step_ch[i] != cur ? kFlush : 0.0);
      if (cost > 0 && cost + add > cap) {
        ++w;
        if (starts) starts->push_back(i);
        cost = 0;
        add = 1.0 + kFlush;
      }
      cost += add;
      cur = step_ch[i];
    }
    return w + 1;
  };
  double lo = 1.0 + kFlush, hi = (double)n * (1.0 + kFlush) + 1.0;
  for (int it = 0; it < 60; ++it) {
    const double mid = 0.5 * (lo + hi);
    if (fill(mid, nullptr) <= NBS_ROW_WARPS) hi = mid; else lo = mid;
  }
  std::vector<int> starts;
  fill(hi, &starts);
  while ((int)starts.size() < NBS_ROW_WARPS) starts.push_back(n);
  starts.push_back(n);
  return starts;  // NBS_ROW_WARPS + 1 step offsets
}

}  // namespace

void build_row_chunks(Plan& plan, int smem_limit) {
  plan.rows_ok = false;
  plan.row_chunks.clear();
  plan.row_aent.clear();
  plan.row_adesc.clear();
  plan.row_rec.clear();
  plan.row_ch.clear();
  plan.row_segs.clear();
  plan.row_scales.clear();
  plan.row_smem = 0;
  std::string why;
  std::vector<double> scales;

  for (const GroupHdr& g : plan.groups) {
    if (g.ncell1 > NBS_ROW_SLAB || g.ncell2 > NBS_ROW_SLAB) {
      plan.row_why = "stored type larger than a slab side";
      return;
    }
    // rows of every term of the group
    std::vector<std::vector<TermRows>> ch_terms(g.nch);
    for (int local = 0; local < g.nch; ++local) {
      const int ci = plan.group_ch[g.ch_off + local];
      for (int t = plan.ch_term_begin[ci]; t < plan.ch_term_begin[ci + 1]; ++t) {
        TermRows tr;
        if (!term_rows(plan, plan.terms[t], g.base1, g.base2, tr, why)) {
          plan.row_why = why;
          return;
        }
        ch_terms[local].push_back(std::move(tr));
      }
    }
    auto ch_steps = [&](int local) {
      int xi = 0;
      const int ci = plan.group_ch[g.ch_off + local];
      for (int t = plan.ch_term_begin[ci]; t < plan.ch_term_begin[ci + 1]; ++t) xi += plan.terms[t].K;
      return (xi + 7) / 8;
    };
    // greedy chunks of whole channels within the shared-memory limit
    int c0 = 0;
    while (c0 < g.nch) {
      SideRows s1, s2;
      int c1 = c0, steps = 0;
      for (; c1 < g.nch; ++c1) {
        SideRows t1 = s1, t2 = s2;
        const int ci = plan.group_ch[g.ch_off + c1];
        for (size_t j = 0; j < ch_terms[c1].size(); ++j) {
          const TermRows& tr = ch_terms[c1][j];
          for (auto& r : tr.r1)
            if (!r.empty) t1.add(r.key);
          for (auto& r : tr.r2)
            if (!r.empty) t2.add(r.key);
        }
        (void)ci;
        const int st = steps + ch_steps(c1);
        const int nch = c1 - c0 + 1;
        const int nrow = (int)std::max<size_t>(t1.keys.size(), 1) + (int)std::max<size_t>(t2.keys.size(), 1);
        const size_t sm = row_chunk_smem(nrow, (int)(t1.entries + t2.entries + 16), st, nch + NBS_ROW_WARPS,
                                         nch + NBS_ROW_WARPS, nch);
        if (c1 > c0 && (sm > (size_t)smem_limit || (int)t1.keys.size() > NBS_ROW_MAX_ROWS ||
                        (int)t2.keys.size() > NBS_ROW_MAX_ROWS))
          break;
        if (sm > (size_t)smem_limit || (int)t1.keys.size() > NBS_ROW_MAX_ROWS ||
            (int)t2.keys.size() > NBS_ROW_MAX_ROWS) {
          plan.row_why = "one channel's rows and records exceed a block's shared memory";
          return;
        }
        // keep the extended sets (rebuild the key pointers into the copies)
        s1 = SideRows();
        s2 = SideRows();
        for (int c = c0; c <= c1; ++c)
          for (auto& tr : ch_terms[c]) {
            for (auto& r : tr.r1)
              if (!r.empty) s1.add(r.key);
            for (auto& r : tr.r2)
              if (!r.empty) s2.add(r.key);
          }
        steps = st;
      }
      // ---- finalise chunk [c0, c1) ----
      RowChunkHdr h = {};
      h.base1 = g.base1;
      h.ncell1 = g.ncell1;
      h.base2 = g.base2;
      h.ncell2 = g.ncell2;
      // row order: longest lists first (warp-uniform trip counts in phase A); an all-zero
      // placeholder row where a side has none
      auto order = [](SideRows& s, std::vector<int>& idx_of) {
        std::vector<int> ord(s.keys.size());
        for (size_t i = 0; i < ord.size(); ++i) ord[i] = (int)i;
        std::stable_sort(ord.begin(), ord.end(),
                         [&](int a, int b) { return s.keys[a]->size() > s.keys[b]->size(); });
        idx_of.assign(ord.size(), 0);
        for (size_t i = 0; i < ord.size(); ++i) idx_of[ord[i]] = (int)i;
        return ord;
      };
      std::vector<int> idx1, idx2;
      const std::vector<int> ord1 = order(s1, idx1), ord2 = order(s2, idx2);
      h.nrow1 = std::max<int>((int)ord1.size(), 1);
      h.nrow2 = std::max<int>((int)ord2.size(), 1);
      h.adesc_off = (int)plan.row_adesc.size();
      h.aent_off = (int)plan.row_aent.size();
      auto emit_rows = [&](SideRows& s, const std::vector<int>& ord) {
        if (ord.empty()) {
          plan.row_adesc.push_back(0u);  // count 0: a zero row
          return;
        }
        for (int r : ord) {
          const RowKey& k = *s.keys[r];
          const unsigned off = (unsigned)(plan.row_aent.size() - h.aent_off);
          plan.row_adesc.push_back(off | (unsigned)k.size() << 20);
          for (auto& e : k) {
            const unsigned code = (e.second < 0 ? 1u : 0u) | (std::abs(e.second) == 2 ? 2u : 0u);
            plan.row_aent.push_back((unsigned short)(e.first | code << 11));
          }
        }
      };
      emit_rows(s1, ord1);
      emit_rows(s2, ord2);
      h.naent = (int)plan.row_aent.size() - h.aent_off;
      while ((plan.row_aent.size() - h.aent_off) % 8) plan.row_aent.push_back(0);
      while ((plan.row_adesc.size() - h.adesc_off) % 4) plan.row_adesc.push_back(0u);
      // records, channel by channel, each padded to whole steps
      h.rec_off = (int)plan.row_rec.size();
      h.ch_off = (int)plan.row_ch.size();
      h.nch = c1 - c0;
      std::vector<int> step_ch;
      for (int c = c0; c < c1; ++c) {
        const int local = c - c0;
        plan.row_ch.push_back(plan.group_ch[g.ch_off + c]);
        long long nrec = 0;
        const int ci = plan.group_ch[g.ch_off + c];
        for (int j = 0; j < (int)ch_terms[c].size(); ++j) {
          const TermHdr& th = plan.terms[plan.ch_term_begin[ci] + j];
          const TermRows& tr = ch_terms[c][j];
          const int nh1 = held_count(th.shape), nh2 = 4 / nh1;
          for (int k = 0; k < th.K; ++k) {
            for (int s = 0; s < 4; ++s) {
              int h1, h2;
              held_of(th.shape, s, h1, h2);
              const RowOf& a = tr.r1[(size_t)k * nh1 + h1];
              const RowOf& b = tr.r2[(size_t)k * nh2 + h2];
              unsigned w = NBS_ROW_SCALES - 1;
              if (!a.empty && !b.empty) {
                const int code = scale_code(scales, tr.m1 * tr.m2 * a.sign * b.sign, why);
                if (code < 0) {
                  plan.row_why = why;
                  return;
                }
                w = (unsigned)code | (unsigned)idx1[s1.id.at(a.key)] << 5 | (unsigned)idx2[s2.id.at(b.key)] << 21;
              }
              plan.row_rec.push_back(w);
            }
            ++nrec;
          }
        }
        while (nrec % 8) {
          for (int s = 0; s < 4; ++s) plan.row_rec.push_back(NBS_ROW_SCALES - 1);
          ++nrec;
        }
        for (long long i = 0; i < nrec / 8; ++i) step_ch.push_back(local);
      }
      h.nstep = (int)step_ch.size();
      // warps and their segments
      const std::vector<int> starts = split_steps(step_ch);
      h.seg_off = (int)plan.row_segs.size();
      int nslot = 0;
      for (int w = 0; w < NBS_ROW_WARPS; ++w) {
        h.seg_base[w] = (int)plan.row_segs.size() - h.seg_off;
        h.out_base[w] = nslot;
        h.cfirst[w] = 0;
        const int a = starts[w], b = starts[w + 1];
        if (a >= b) continue;
        h.cfirst[w] = step_ch[a];
        for (int i = a; i < b;) {
          int j = i;
          while (j < b && step_ch[j] == step_ch[i]) ++j;
          plan.row_segs.push_back({i, j, step_ch[i], 0});
          i = j;
        }
        nslot += step_ch[b - 1] - step_ch[a] + 1;
      }
      h.seg_base[NBS_ROW_WARPS] = (int)plan.row_segs.size() - h.seg_off;
      h.out_base[NBS_ROW_WARPS] = nslot;
      h.nslot = nslot;
      h.smem = (int)row_chunk_smem(h.nrow1 + h.nrow2, h.naent, h.nstep, h.nslot, h.seg_base[NBS_ROW_WARPS], h.nch);
      if (h.smem > smem_limit) {
        plan.row_why = "a chunk exceeds a block's shared memory";
        return;
      }
      plan.row_smem = std::max(plan.row_smem, h.smem);
      plan.row_chunks.push_back(h);
      c0 = c1;
    }
  }
  plan.row_scales.assign(NBS_ROW_SCALES, 0.0);
  for (size_t i = 0; i < scales.size(); ++i) plan.row_scales[i] = scales[i];
  plan.rows_ok = !plan.row_chunks.empty();
  if (!plan.rows_ok) plan.row_why = "no chunks";
}

}  // namespace nbs
