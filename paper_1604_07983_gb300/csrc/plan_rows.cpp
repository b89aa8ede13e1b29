// plan_rows.cpp -- tables of the two-phase contraction (kernels_rows.cu).
//
// The gather lists of the effective blocks (Eq. (4.2); Sec. 4 (ii)) repeat
// heavily across terms and channels: over the 52 channels about 87 thousand
// (shared index, held spin) rows of each side are built from only a few
// thousand distinct sums of stored cells.  So every distinct row is listed
// once (phase A builds it per momentum for all four sink spins), and the
// product of Eq. (4.3) walks records that name, for each shared index xi~ and
// output source-spin pair s, the row of each side and a scale (phase B); the
// products of a channel that name the same two rows for the same s are merged
// into one record with the sum of their scales.
//
// A row is kept up to a scale: with m the smallest coefficient magnitude of
// its term side, its coefficients are m times +-1 or +-2, and it is stored
// with the sign that makes its first entry (lowest cell) positive.  The
// product's scale is then m1 m2 sign1 sign2; a record's scale, the sum over
// the products it merges, is one of at most 63 values over a plan (a code
// into Plan::row_scales).
//
// Over all channels the rows depend only on the stored type they sum, so the
// rows of each type are listed once (Plan::row_types, row_desc, row_ent: the
// effective-block kernel builds them for every momentum) and each chunk's
// records name rows of its two types.
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

using RowKey = std::vector<std::pair<int, int>>;  // (cell of the stored type, integer coefficient), cells ascending

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
          if (cell < 0 || cell >= 4096) {
            why = "cell outside its stored type or beyond 4096";
            return false;
          }
          r.key.push_back({cell, iq});
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
    why = "more than 63 distinct product scales";
    return -1;
  }
  scales.push_back(v);
  return (int)scales.size() - 1;
}

// contiguous split of the chunk's steps into NBS_ROW_WARPS ranges: a warp's
// cost is its steps plus kFlush per segment (a run of one key) it holds; bisection on the
// largest cost, greedy fill
constexpr double kFlush = 2.0;

std::vector<int> split_steps(const std::vector<int>& step_ch) {  // a flush where the key changes
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

// Greedy colouring of one stored type's rows (provisional ids 0..n-1) with 8 colours so that the distinct
// rows one warp loads in a step (its 32 records: B1's rows, or B2's) spread evenly over the 8 16-byte bank
// groups (row mod 8), over every chunk that reads the type (srcs: a chunk's records and the side on which
// it reads the type): rows in order of their co-load count, each taking the colour least shared with its
// coloured co-loads (ties: the least used colour).  idx[r] = colour + 8 * (rank within the colour);
// npad = 8 * largest class.
template <typename PRecT>
void color_rows(const std::vector<std::pair<const std::vector<PRecT>*, int>>& srcs, int n, std::vector<int>& idx,
                int& npad) {
  std::vector<std::map<int, int>> adj(n);
  for (const auto& src : srcs) {
    const std::vector<PRecT>& prec = *src.first;
    const int side = src.second;
    const size_t nq = prec.size() / 8;  // quarter-warps: lanes 8 q .. 8 q + 7 of a warp step
    for (size_t qi = 0; qi < nq; ++qi) {
      int rows[8], m = 0;
      for (int j = 0; j < 8; ++j) {
        const PRecT& r = prec[qi * 8 + j];
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
  }
  std::vector<int> order(n), weight(n, 0), color(n, -1);
  for (int r = 0; r < n; ++r) {
    order[r] = r;
    for (auto& kv : adj[r]) weight[r] += kv.second;
  }
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return weight[a] > weight[b]; });
  int used[8] = {};
  const int cap = (n + 7) / 8 + 1;  // classes stay within one row of even: padding rows cost bytes and room
  for (int r : order) {
    long long cost[8] = {};
    for (auto& kv : adj[r])
      if (color[kv.first] >= 0) cost[color[kv.first]] += kv.second;
    int best = -1;
    for (int c = 0; c < 8; ++c)
      if (used[c] < cap &&
          (best < 0 || cost[c] < cost[best] || (cost[c] == cost[best] && used[c] < used[best])))
        best = c;
    color[r] = best;
    ++used[best];
  }
  int rank[8] = {}, big = 0;
  idx.assign(n, 0);
  for (int r = 0; r < n; ++r) idx[r] = color[r] + 8 * rank[color[r]]++;
  for (int c = 0; c < 8; ++c) big = std::max(big, used[c]);
  npad = std::max(8, 8 * big);
}

// The records of one (channel, s) list, regrouped over the list's quarters (the eight lanes of one lane
// group in one warp step): a 16-byte shared-memory load of a warp is served in four phases of eight lanes,
// and a phase takes as many wavefronts as its fullest 16-byte bank group (row mod 8) has distinct rows.
// Each quarter is filled greedily with the records that add no second row to a bank group on either side
// (a row already in the quarter adds none), preferring the records whose bank groups are the most common
// among those left; every quarter but the list's last stays full.
template <typename PRecT>
void regroup_quarters(std::vector<PRecT>& prec, const std::vector<size_t>& qs, const std::vector<int>& idx1,
                      const std::vector<int>& idx2) {
  std::vector<PRecT> pool;
  for (size_t b : qs)
    for (int k = 0; k < 8; ++k)
      if (prec[b + k].r1 >= 0) pool.push_back(prec[b + k]);
  int cnt1[8] = {}, cnt2[8] = {};
  for (const PRecT& r : pool) {
    ++cnt1[idx1[r.r1] & 7];
    ++cnt2[idx2[r.r2] & 7];
  }
  std::vector<char> used(pool.size(), 0);
  size_t left = pool.size();
  for (size_t b : qs) {
    int row1[8], row2[8];
    for (int c = 0; c < 8; ++c) row1[c] = row2[c] = -1;
    for (int k = 0; k < 8; ++k) {
      PRecT pick = {NBS_ROW_SCALES - 1, -1, -1};
      if (left) {
        long best = -1;
        int bpen = 0, bab = 0;
        for (size_t j = 0; j < pool.size(); ++j) {
          if (used[j]) continue;
          const int c1 = idx1[pool[j].r1] & 7, c2 = idx2[pool[j].r2] & 7;
          const int pen = (row1[c1] >= 0 && row1[c1] != pool[j].r1) + (row2[c2] >= 0 && row2[c2] != pool[j].r2);
          const int ab = cnt1[c1] + cnt2[c2];
          if (best < 0 || pen < bpen || (pen == bpen && ab > bab)) {
            best = (long)j;
            bpen = pen;
            bab = ab;
          }
        }
        used[best] = 1;
        --left;
        pick = pool[best];
        const int c1 = idx1[pick.r1] & 7, c2 = idx2[pick.r2] & 7;
        --cnt1[c1];
        --cnt2[c2];
        if (row1[c1] < 0) row1[c1] = pick.r1;
        if (row2[c2] < 0) row2[c2] = pick.r2;
      }
      prec[b + k] = pick;
    }
  }
}

// One attempt at the row tables: chunks are cut with each type's rows estimated as its distinct rows
// (rounded up to 8) plus `margin`, the room its bank colouring may add.
void build_rows_once(Plan& plan, int smem_limit, int margin) {
  plan.rows_ok = false;
  plan.row_types.clear();
  plan.row_desc.clear();
  plan.row_ent.clear();
  plan.row_nr = 0;
  plan.row_chunks.clear();
  plan.row_rec.clear();
  plan.row_ch.clear();
  plan.row_segs.clear();
  plan.row_scales.clear();
  plan.row_smem = 0;
  std::string why;
  std::vector<double> scales;

  // ---- the rows of every term of every group, and the distinct rows of each stored type ----
  std::map<int, int> type_of;  // stored type's first cell -> row type
  std::vector<SideRows> trows;
  std::vector<int> tncell;
  auto type_index = [&](int base, int ncell) {
    auto it = type_of.find(base);
    if (it != type_of.end()) return it->second;
    const int t = (int)trows.size();
    type_of[base] = t;
    trows.emplace_back();
    tncell.push_back(ncell);
    return t;
  };
  std::vector<std::vector<std::vector<TermRows>>> g_terms(plan.groups.size());
  for (size_t gi = 0; gi < plan.groups.size(); ++gi) {
    const GroupHdr& g = plan.groups[gi];
    const int t1 = type_index(g.base1, g.ncell1), t2 = type_index(g.base2, g.ncell2);
    g_terms[gi].resize(g.nch);
    for (int local = 0; local < g.nch; ++local) {
      const int ci = plan.group_ch[g.ch_off + local];
      for (int t = plan.ch_term_begin[ci]; t < plan.ch_term_begin[ci + 1]; ++t) {
        TermRows tr;
        if (!term_rows(plan, plan.terms[t], g.base1, g.base2, tr, why)) {
          plan.row_why = why;
          return;
        }
        for (auto& r : tr.r1)
          if (!r.empty) trows[t1].add(r.key);
        for (auto& r : tr.r2)
          if (!r.empty) trows[t2].add(r.key);
        g_terms[gi][local].push_back(std::move(tr));
      }
    }
  }
  const int ntypes = (int)trows.size();
  if (ntypes > 8) {
    plan.row_why = "more than 8 stored types";
    return;
  }
  // row counts after the bank colouring, estimated (8 colour classes of nearly equal size)
  std::vector<int> nrow_est(ntypes);
  for (int t = 0; t < ntypes; ++t) {
    nrow_est[t] = (int)(trows[t].keys.size() + 7) / 8 * 8 + margin;
    if ((int)trows[t].keys.size() > NBS_ROW_MAX_ROWS) {
      plan.row_why = "more than 4095 distinct rows of one stored type";
      return;
    }
  }

  // ---- chunks of whole channels of one group within the shared-memory limit; records with provisional
  // row ids (the types' insertion order), each channel padded to whole steps; -1 marks no product ----
  struct PRec { int code, r1, r2; };
  struct ChunkBuild {
    RowChunkHdr h;
    std::vector<PRec> prec;
    std::vector<int> step_ch;   // chunk-local channel of each step
    std::vector<int> step_map;  // its lane-group map: the s of group g in bits 2 g, 2 g + 1
    std::vector<std::vector<size_t>> list_q;  // per (channel, s) list: the first record of each of its quarters
  };
  std::vector<ChunkBuild> cbs;
  for (size_t gi = 0; gi < plan.groups.size(); ++gi) {
    const GroupHdr& g = plan.groups[gi];
    const int t1 = type_of.at(g.base1), t2 = type_of.at(g.base2);
    int c0 = 0;
    while (c0 < g.nch) {
      int c1 = c0 + 1;
      for (; c1 < g.nch; ++c1) {  // take channel c1 as well?
        const int nch = c1 - c0 + 1;
        if (row_chunk_smem(nrow_est[t1], nrow_est[t2], nch + NBS_ROW_WARPS, 4 * nch + NBS_ROW_WARPS, nch) >
            (size_t)smem_limit)
          break;
      }
      if (row_chunk_smem(nrow_est[t1], nrow_est[t2], 1 + NBS_ROW_WARPS, 4 + NBS_ROW_WARPS, 1) > (size_t)smem_limit) {
        plan.row_why = "one channel's rows exceed a block's shared memory";
        return;
      }
      ChunkBuild cb;
      RowChunkHdr& h = cb.h;
      h = RowChunkHdr();
      h.type1 = t1;
      h.type2 = t2;
      h.ch_off = (int)plan.row_ch.size();
      h.nch = c1 - c0;
      for (int c = c0; c < c1; ++c) {
        const int local = c - c0;
        const int ci = plan.group_ch[g.ch_off + c];
        plan.row_ch.push_back(ci);
        // the channel's products, merged: for each output pair s, every (B1 row, B2 row) the terms name
        // once, with the sum of their scales (products whose scales cancel are dropped) -- the same sum of
        // Eq. (4.3), term by term, regrouped by the rows it multiplies
        std::map<std::pair<int, int>, double> merged[4];
        double smax = 0;
        for (int j = 0; j < (int)g_terms[gi][c].size(); ++j) {
          const TermHdr& th = plan.terms[plan.ch_term_begin[ci] + j];
          const TermRows& tr = g_terms[gi][c][j];
          const int nh1 = held_count(th.shape), nh2 = 4 / nh1;
          for (int k = 0; k < th.K; ++k)
            for (int s = 0; s < 4; ++s) {
              int h1, h2;
              held_of(th.shape, s, h1, h2);
              const RowOf& a = tr.r1[(size_t)k * nh1 + h1];
              const RowOf& b = tr.r2[(size_t)k * nh2 + h2];
              if (a.empty || b.empty) continue;
              const double v = tr.m1 * tr.m2 * a.sign * b.sign;
              merged[s][{trows[t1].id.at(a.key), trows[t2].id.at(b.key)}] += v;
              smax = std::max(smax, std::fabs(v));
            }
        }
        // lane groups: lane 8 g + kq is in group g; a group takes eight records of one s per step, so that
        // the list of s is cut into ceil(n_s / 8) group-steps.  The channel's group-steps (s = 0, 1, 2, 3 in
        // turn) fill the four groups one after the other, H = ceil(total / 4) each, so that the lists of
        // unequal length share the steps; a step's map names the s of each group (bits 2 g, 2 g + 1)
        std::vector<PRec> lists[4];
        std::vector<std::pair<int, size_t>> gs;  // (s, first record) of each group-step
        for (int s = 0; s < 4; ++s) {
          for (auto& kv : merged[s]) {
            if (std::fabs(kv.second) <= 1e-12 * smax) continue;  // the terms' scales cancel
            PRec r = {scale_code(scales, kv.second, why), kv.first.first, kv.first.second};
            if (r.code < 0) {
              plan.row_why = why;
              return;
            }
            lists[s].push_back(r);
          }
          for (size_t k = 0; k < lists[s].size(); k += 8) gs.push_back({s, k});
        }
        const size_t H = (gs.size() + 3) / 4;
        std::vector<size_t> qpos[4];
        for (size_t e = 0; e < gs.size(); ++e)
          qpos[gs[e].first].push_back(((cb.step_ch.size() + e % H) * 4 + e / H) * 8);
        for (int s = 0; s < 4; ++s)
          if (!qpos[s].empty()) cb.list_q.push_back(std::move(qpos[s]));
        for (size_t st = 0; st < H; ++st) {
          int map = 0;
          for (int g = 0; g < 4; ++g) {
            // a group past its last group-step keeps the s of its last one (padding records), so that
            // its map does not change
            const size_t e = (size_t)g * H + st;
            const size_t last = std::min(gs.size(), (size_t)(g + 1) * H);
            const int sg = e < last ? gs[e].first : ((size_t)g * H < last ? gs[last - 1].first : 0);
            map |= sg << (2 * g);
          }
          for (int g = 0; g < 4; ++g)
            for (int kq = 0; kq < 8; ++kq) {
              const size_t e = (size_t)g * H + st;
              PRec r = {NBS_ROW_SCALES - 1, -1, -1};
              if (e < std::min(gs.size(), (size_t)(g + 1) * H)) {
                const size_t k = gs[e].second + (size_t)kq;
                if (k < lists[gs[e].first].size()) r = lists[gs[e].first][k];
              }
              cb.prec.push_back(r);
            }
          cb.step_ch.push_back(local);
          cb.step_map.push_back(map);
        }
      }
      cbs.push_back(std::move(cb));
      c0 = c1;
    }
  }

  // largest chunks first: within each momentum block the product kernel's blocks start in this order, so
  // the launch ends on the shortest blocks
  std::stable_sort(cbs.begin(), cbs.end(), [](const ChunkBuild& a, const ChunkBuild& b) {
    return a.step_ch.size() > b.step_ch.size();
  });

  // ---- row numbers per type: bank colouring over every chunk that reads the type ----
  std::vector<std::vector<int>> idx(ntypes);
  int roff = 0;
  for (int t = 0; t < ntypes; ++t) {
    std::vector<std::pair<const std::vector<PRec>*, int>> srcs;
    for (const ChunkBuild& cb : cbs) {
      if (cb.h.type1 == t) srcs.push_back({&cb.prec, 0});
      if (cb.h.type2 == t) srcs.push_back({&cb.prec, 1});
    }
    int npad = 0;
    color_rows(srcs, (int)trows[t].keys.size(), idx[t], npad);
    // within each colour, rows numbered by decreasing entry count: the eight rows of an octet (one of each
    // colour) that the row kernel builds side by side then have similar counts
    {
      std::vector<int> byc[8];
      for (int i = 0; i < (int)idx[t].size(); ++i) byc[idx[t][i] & 7].push_back(i);
      for (int c = 0; c < 8; ++c) {
        std::stable_sort(byc[c].begin(), byc[c].end(), [&](int a, int b) {
          return trows[t].keys[a]->size() > trows[t].keys[b]->size();
        });
        for (size_t k = 0; k < byc[c].size(); ++k) idx[t][byc[c][k]] = c + 8 * (int)k;
      }
    }
    if (npad > NBS_ROW_MAX_ROWS) {
      plan.row_why = "too many rows after bank colouring";
      return;
    }
    RowTypeHdr th = {};
    th.base = -1;
    for (auto& kv : type_of)
      if (kv.second == t) th.base = kv.first;
    th.ncell = tncell[t];
    th.roff = roff;
    th.nrow = npad;
    plan.row_types.push_back(th);
    roff += npad;
  }
  plan.row_nr = roff;
  // row descriptors and entries in row order (padding rows have no entries)
  plan.row_desc.assign((size_t)roff, 0u);
  for (int t = 0; t < ntypes; ++t) {
    const RowTypeHdr& th = plan.row_types[t];
    std::vector<int> by_row(th.nrow, -1);
    for (int i = 0; i < (int)trows[t].keys.size(); ++i) by_row[idx[t][i]] = i;
    for (int r = 0; r < th.nrow; ++r) {
      const unsigned off = (unsigned)plan.row_ent.size();
      unsigned cnt = 0;
      if (by_row[r] >= 0) {
        const RowKey& k = *trows[t].keys[by_row[r]];
        if (k.size() >= 32) {
          plan.row_why = "a row of 32 or more entries";
          return;
        }
        for (auto& e : k) {
          const unsigned code = (e.second < 0 ? 1u : 0u) | (std::abs(e.second) == 2 ? 2u : 0u);
          plan.row_ent.push_back((unsigned short)((unsigned)e.first | code << 12));
        }
        cnt = (unsigned)k.size();
      }
      if (off >= (1u << 24)) {
        plan.row_why = "row entry table beyond its descriptor field";
        return;
      }
      plan.row_desc[(size_t)th.roff + r] = off | cnt << 24 | (unsigned)t << 29;
    }
  }

  // ---- each list's records regrouped over its quarters (final row numbers known) ----
  for (ChunkBuild& cb : cbs)
    for (const std::vector<size_t>& qs : cb.list_q) regroup_quarters(cb.prec, qs, idx[cb.h.type1], idx[cb.h.type2]);

  // ---- chunks: final records, warp ranges and segments, shared memory ----
  for (ChunkBuild& cb : cbs) {
    RowChunkHdr h = cb.h;
    const RowTypeHdr &A = plan.row_types[h.type1], &B = plan.row_types[h.type2];
    h.roff1 = A.roff;
    h.nrow1 = A.nrow;
    h.roff2 = B.roff;
    h.nrow2 = B.nrow;
    h.rec_off = (int)plan.row_rec.size();
    for (const PRec& r : cb.prec) {
      if (r.r1 < 0) plan.row_rec.push_back((unsigned)(NBS_ROW_SCALES - 1) << 24);
      else
        plan.row_rec.push_back((unsigned)idx[h.type1][r.r1] | (unsigned)idx[h.type2][r.r2] << 12 |
                               (unsigned)r.code << 24);
    }
    h.nstep = (int)cb.step_ch.size();
    // a warp flushes where the channel or the group map changes
    std::vector<int> key(cb.step_ch.size());
    for (size_t i = 0; i < key.size(); ++i) key[i] = cb.step_ch[i] << 8 | cb.step_map[i];
    const std::vector<int> starts = split_steps(key);
    h.seg_off = (int)plan.row_segs.size();
    int nslot = 0;
    for (int w = 0; w < NBS_ROW_WARPS; ++w) {
      h.seg_base[w] = (int)plan.row_segs.size() - h.seg_off;
      h.out_base[w] = nslot;
      h.cfirst[w] = 0;
      const int a = starts[w], b = starts[w + 1];
      if (a >= b) continue;
      h.cfirst[w] = cb.step_ch[a];
      for (int i = a; i < b;) {
        int j = i;
        while (j < b && key[j] == key[i]) ++j;
        // the group map, each group's rank among the groups of its s (bits 8 + 2 g), and the number of
        // groups that share the most common s (bits 16..18): the flush adds the groups in that many turns
        const int m = cb.step_map[i];
        int word = m, passes = 1;
        for (int g = 0; g < 4; ++g) {
          int rank = 0;
          for (int h = 0; h < g; ++h) rank += ((m >> (2 * h)) & 3) == ((m >> (2 * g)) & 3);
          word |= rank << (8 + 2 * g);
          passes = std::max(passes, rank + 1);
        }
        plan.row_segs.push_back({i, j, cb.step_ch[i], word | passes << 16});
        i = j;
      }
      nslot += cb.step_ch[b - 1] - cb.step_ch[a] + 1;
    }
    h.seg_base[NBS_ROW_WARPS] = (int)plan.row_segs.size() - h.seg_off;
    h.out_base[NBS_ROW_WARPS] = nslot;
    h.nslot = nslot;
    h.smem = (int)row_chunk_smem(h.nrow1, h.nrow2, h.nslot, h.seg_base[NBS_ROW_WARPS], h.nch);
    if (h.smem > smem_limit) {
      plan.row_why = "a chunk exceeds a block's shared memory";
      return;
    }
    plan.row_smem = std::max(plan.row_smem, h.smem);
    plan.row_chunks.push_back(h);
  }
  // the kernel reads each warp's records a few steps ahead of use: padding steps after the last chunk
  plan.row_rec.insert(plan.row_rec.end(), 4 * 32, (unsigned)(NBS_ROW_SCALES - 1) << 24);
  plan.row_scales.assign(NBS_ROW_SCALES, 0.0);
  for (size_t i = 0; i < scales.size(); ++i) plan.row_scales[i] = scales[i];
  plan.rows_ok = !plan.row_chunks.empty();
  if (!plan.rows_ok) plan.row_why = "no chunks";
}

}  // namespace

void build_row_chunks(Plan& plan, int smem_limit) {
  // a chunk cut on too small an estimate of its rows can exceed the limit once its rows are numbered:
  // cut again with more room
  for (int margin = 32; margin <= 512; margin *= 2) {
    build_rows_once(plan, smem_limit, margin);
    if (plan.rows_ok || plan.row_why != "a chunk exceeds a block's shared memory") return;
  }
}

}  // namespace nbs
