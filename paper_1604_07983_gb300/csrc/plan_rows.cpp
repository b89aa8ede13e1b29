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

// 16-byte unit of sink spins 0, 1 of cell `cell` of slab side `side` in the kernel's planar slab: each
// side is four TMA boxes of NBS_ROW_BOX cells, a box holding spins 0, 1 of its cells, then spins 2, 3
// (the unit of spins 2, 3 is NBS_ROW_BOX further)
int slab_unit(int side, int cell) {
  return side * 2 * NBS_ROW_SLAB + (cell / NBS_ROW_BOX) * 2 * NBS_ROW_BOX + cell % NBS_ROW_BOX;
}

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
    const int base = side ? base2 : base1;
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
          r.key.push_back({slab_unit(side, cell), iq});
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
  // spread: warp w takes steps while its cost stays within both the smallest feasible largest cost and
  // the remaining cost divided by the remaining warps (rounded up to a whole step), so that no warp idles
  // while another holds the largest share
  double total = 0;
  for (int i = n - 1; i >= 0; --i) total += 1.0 + ((i == 0 || step_ch[i] != step_ch[i - 1]) ? kFlush : 0.0);
  std::vector<int> starts(1, 0);
  int i = 0;
  double left = total;
  for (int w = 0; w < NBS_ROW_WARPS; ++w) {
    const double target = std::min(hi, left / (NBS_ROW_WARPS - w) + 1.0);
    double cost = 0;
    int cur = -1;
    while (i < n) {
      const double add = 1.0 + (step_ch[i] != cur ? kFlush : 0.0);
      if (cost > 0 && cost + add > target) break;
      cost += add;
      cur = step_ch[i];
      ++i;
    }
    left = std::max(0.0, left - cost);
    starts.push_back(i);
  }
  if (i < n) {  // fall back to the greedy fill at the feasible cap
    starts.clear();
    fill(hi, &starts);
    while ((int)starts.size() < NBS_ROW_WARPS) starts.push_back(n);
    starts.push_back(n);
  }
  return starts;  // NBS_ROW_WARPS + 1 step offsets
}

// Greedy colouring of one side's rows (provisional ids 0..n-1) with 8 colours so that the distinct rows
// one warp loads in a step (its 32 records) spread evenly over the 8 16-byte bank groups (row mod 8):
// rows in order of their co-load count, each taking the colour least shared with its coloured co-loads
// (ties: the least used colour).  idx[r] = colour + 8 * (rank within the colour); npad = 8 * largest
// class.
template <typename PRecT>
void color_rows(const std::vector<PRecT>& prec, int n, int side, std::vector<int>& idx, int& npad) {
  std::vector<std::map<int, int>> adj(n);
  const size_t nq = prec.size() / 32;  // warp steps of 32 records
  for (size_t qi = 0; qi < nq; ++qi) {
    int rows[32], m = 0;
    for (int j = 0; j < 32; ++j) {
      const PRecT& r = prec[qi * 32 + j];
      const int id = side ? r.r2 : r.r1;
      if (id < 0) continue;
      bool dup = false;
      for (int i = 0; i < m; ++i) dup = dup || rows[i] == id;
      if (!dup) rows[m++] = id;
    }
    for (int a = 0; a < m; ++a)
      for (int b = 0; b < m; ++b)
        if (a != b) ++adj[rows[a]][rows[b]];
  }
  std::vector<int> order(n), weight(n, 0), color(n, -1);
  for (int r = 0; r < n; ++r) {
    order[r] = r;
    for (auto& kv : adj[r]) weight[r] += kv.second;
  }
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return weight[a] > weight[b]; });
  int used[8] = {};
  for (int r : order) {
    long long cost[8] = {};
    for (auto& kv : adj[r])
      if (color[kv.first] >= 0) cost[color[kv.first]] += kv.second;
    int best = 0;
    for (int c = 1; c < 8; ++c)
      if (cost[c] < cost[best] || (cost[c] == cost[best] && used[c] < used[best])) best = c;
    color[r] = best;
    ++used[best];
  }
  int rank[8] = {}, big = 0;
  idx.assign(n, 0);
  for (int r = 0; r < n; ++r) idx[r] = color[r] + 8 * rank[color[r]]++;
  for (int c = 0; c < 8; ++c) big = std::max(big, used[c]);
  npad = std::max(8, 8 * big);
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
        // the bank colouring pads each side's rows to 8 equal colour classes: allow for it
        const int nd = (int)(t1.keys.size() + t2.keys.size());
        const int nrow = (int)(1.1 * (double)nd) + 32;
        // two row buffers where they fit, else one (a channel alone may need one)
        const int ne = (int)(t1.entries + t2.entries + 16);
        size_t sm = row_chunk_smem(2, nrow, nd, ne, nch + NBS_ROW_WARPS, nch + NBS_ROW_WARPS, nch);
        if (sm > (size_t)smem_limit && c1 == c0)
          sm = row_chunk_smem(1, nrow, nd, ne, nch + NBS_ROW_WARPS, nch + NBS_ROW_WARPS, nch);
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
      // records with provisional row ids (insertion order of s1, s2), channel by channel, each padded
      // to whole steps; -1 marks a record with no product
      struct PRec { int code, r1, r2; };
      std::vector<PRec> prec;
      std::vector<int> step_ch;
      h.ch_off = (int)plan.row_ch.size();
      h.nch = c1 - c0;
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
              PRec r = {NBS_ROW_SCALES - 1, -1, -1};
              if (!a.empty && !b.empty) {
                r.code = scale_code(scales, tr.m1 * tr.m2 * a.sign * b.sign, why);
                if (r.code < 0) {
                  plan.row_why = why;
                  return;
                }
                r.r1 = s1.id.at(a.key);
                r.r2 = s2.id.at(b.key);
              }
              prec.push_back(r);
            }
            ++nrec;
          }
        }
        while (nrec % 8) {
          for (int s = 0; s < 4; ++s) prec.push_back({NBS_ROW_SCALES - 1, -1, -1});
          ++nrec;
        }
        for (long long i = 0; i < nrec / 8; ++i) step_ch.push_back(local);
      }
      // row numbers: the eight rows a quarter warp reads in one 16-byte load (steps of eight shared
      // indices, lanes 4 kq + s, quarter p = kq >> 1) should fall in different 16-byte bank groups,
      // i.e. differ mod 8 (planar row halves); greedy colouring with 8 colours, then row = colour + 8 k
      std::vector<int> idx1, idx2;
      int nr1p = 0, nr2p = 0;
      color_rows(prec, (int)s1.keys.size(), 0, idx1, nr1p);
      color_rows(prec, (int)s2.keys.size(), 1, idx2, nr2p);
      if (nr1p > NBS_ROW_MAX_ROWS || nr2p > NBS_ROW_MAX_ROWS) {
        plan.row_why = "too many rows after bank colouring";
        return;
      }
      h.nrow1 = nr1p;
      h.nrow2 = nr2p;
      h.rec_off = (int)plan.row_rec.size();
      for (const PRec& r : prec) {
        if (r.r1 < 0) plan.row_rec.push_back((unsigned)(NBS_ROW_SCALES - 1) << 24);
        else plan.row_rec.push_back((unsigned)idx1[r.r1] | (unsigned)idx2[r.r2] << 12 | (unsigned)r.code << 24);
      }
      // phase-A descriptors, longest lists first (warp-uniform trip counts): entry offset | count << 14 |
      // target row << 19 (B2's rows after B1's nrow1)
      h.adesc_off = (int)plan.row_adesc.size();
      h.aent_off = (int)plan.row_aent.size();
      std::vector<std::pair<int, int>> all;  // (side, provisional id)
      for (int i = 0; i < (int)s1.keys.size(); ++i) all.push_back({0, i});
      for (int i = 0; i < (int)s2.keys.size(); ++i) all.push_back({1, i});
      // longest lists first (warp-uniform trip counts); within one length, batches of 32 rows (one warp
      // instruction) picked greedily so that their store targets (row slot mod 8) and, for each entry
      // position, their slab units (mod 8) spread over the 16-byte bank groups
      auto target_of = [&](const std::pair<int, int>& x) {
        return x.first ? nr1p + idx2[x.second] : idx1[x.second];
      };
      auto key_of = [&](const std::pair<int, int>& x) -> const RowKey& { return *(x.first ? s2 : s1).keys[x.second]; };
      std::stable_sort(all.begin(), all.end(), [&](const std::pair<int, int>& x, const std::pair<int, int>& y) {
        return key_of(x).size() > key_of(y).size();
      });
      {
        std::vector<std::pair<int, int>> ordered;
        ordered.reserve(all.size());
        for (size_t i = 0; i < all.size();) {
          size_t j = i;
          while (j < all.size() && key_of(all[j]).size() == key_of(all[i]).size()) ++j;
          std::vector<char> taken(j - i, 0);
          size_t left = j - i, first = i;
          while (left) {
            int tc[8] = {}, gc[32][8] = {};
            for (int pick = 0; pick < 32 && left; ++pick) {
              while (taken[first - i]) ++first;
              long best = -1, bestcost = 0;
              int scanned = 0;
              // quadratic in the bank-group counts: a load takes as many wavefronts as its fullest group
              for (size_t k = first; k < j && scanned < 256; ++k) {
                if (taken[k - i]) continue;
                ++scanned;
                const RowKey& kk = key_of(all[k]);
                const int t = tc[target_of(all[k]) & 7];
                long cost = 2L * (2 * t + 1);
                for (size_t e = 0; e < kk.size() && e < 32; ++e) cost += 2 * gc[e][kk[e].first & 7] + 1;
                if (best < 0 || cost < bestcost) { best = (long)k; bestcost = cost; }
              }
              taken[best - i] = 1;
              --left;
              const RowKey& kk = key_of(all[best]);
              ++tc[target_of(all[best]) & 7];
              for (size_t e = 0; e < kk.size() && e < 32; ++e) ++gc[e][kk[e].first & 7];
              ordered.push_back(all[best]);
            }
          }
          i = j;
        }
        all.swap(ordered);
      }
      h.nadesc = (int)all.size();
      for (auto& r : all) {
        const RowKey& k = *(r.first ? s2 : s1).keys[r.second];
        const unsigned off = (unsigned)(plan.row_aent.size() - h.aent_off);
        const unsigned target = r.first ? (unsigned)(nr1p + idx2[r.second]) : (unsigned)idx1[r.second];
        if (off >= (1u << 14) || k.size() >= 32) {
          plan.row_why = "row entry table of a chunk beyond its descriptor fields";
          return;
        }
        plan.row_adesc.push_back(off | (unsigned)k.size() << 14 | target << 19);
        for (auto& e : k) {
          const unsigned code = (e.second < 0 ? 1u : 0u) | (std::abs(e.second) == 2 ? 2u : 0u);
          plan.row_aent.push_back((unsigned short)(e.first | code << 12));
        }
      }
      h.naent = (int)plan.row_aent.size() - h.aent_off;
      while ((plan.row_aent.size() - h.aent_off) % 8) plan.row_aent.push_back(0);
      while ((plan.row_adesc.size() - h.adesc_off) % 4) plan.row_adesc.push_back(0u);
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
      h.nbuf = 2;
      h.smem = (int)row_chunk_smem(2, h.nrow1 + h.nrow2, h.nadesc, h.naent, h.nslot, h.seg_base[NBS_ROW_WARPS], h.nch);
      if (h.smem > smem_limit) {
        h.nbuf = 1;
        h.smem =
            (int)row_chunk_smem(1, h.nrow1 + h.nrow2, h.nadesc, h.naent, h.nslot, h.seg_base[NBS_ROW_WARPS], h.nch);
      }
      if (h.smem > smem_limit) {
        plan.row_why = "a chunk exceeds a block's shared memory";
        return;
      }
      plan.row_smem = std::max(plan.row_smem, h.smem);
      plan.row_chunks.push_back(h);
      c0 = c1;
    }
  }
  // the kernel reads each warp's records a few steps ahead of use: padding steps after the last chunk
  plan.row_rec.insert(plan.row_rec.end(), 4 * 32, (unsigned)(NBS_ROW_SCALES - 1) << 24);
  plan.row_scales.assign(NBS_ROW_SCALES, 0.0);
  for (size_t i = 0; i < scales.size(); ++i) plan.row_scales[i] = scales[i];
  plan.rows_ok = !plan.row_chunks.empty();
  if (!plan.rows_ok) plan.row_why = "no chunks";
}

}  // namespace nbs
