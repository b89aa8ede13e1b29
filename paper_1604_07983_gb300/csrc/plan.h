// plan.h -- host-side channel compiler: Wick topologies -> gather tables.
//
// The classification of the Wick contractions into effective-block terms is
// done once on the CPU and packed as structures of arrays for the device
// (Sec. 4 (ii)-(iii) of arXiv:1604.07983).
#pragma once
#include <string>
#include <vector>

namespace nbs {

enum Flavour { FU = 0, FD = 1, FS = 2 };
enum Field { P = 0, N, SIGP, SIG0, SIGM, XI0, XIM, LAM, XU, XD, XS, NFIELDS };
// normal-block flavour patterns (u = d = l): q1 q2 q3
// Normal-block patterns: pattern = diquark * nflav + flavour of the third
// quark, the diquark being an ordered flavour pair of the propagators in use.
// nflav = 2 (u = d = l, s): diquarks ll, ls -> patterns lll, lls, lsl, lss;
// nflav = 3 (u, d, s):      diquarks uu, ud, dd, us, ds -> 15 patterns.
enum Pattern { LLL = 0, LLS = 1, LSL = 2, LSS = 3 };
#define NBS_MAX_DIQUARKS 5
inline int n_diquarks(int nflav) { return nflav == 2 ? 2 : 5; }
// flavours (f0 <= f1) of diquark d; -1 if d is out of range
inline void diquark_flavours(int nflav, int d, int& f0, int& f1) {
  static const int p2[2][2] = {{0, 0}, {0, 1}};
  static const int p3[5][2] = {{0, 0}, {0, 1}, {1, 1}, {0, 2}, {1, 2}};
  if (nflav == 2 && d >= 0 && d < 2) { f0 = p2[d][0]; f1 = p2[d][1]; return; }
  if (nflav == 3 && d >= 0 && d < 5) { f0 = p3[d][0]; f1 = p3[d][1]; return; }
  f0 = f1 = -1;
}

struct Mono { double c; int q[3]; };
const std::vector<Mono>& field_monomials(int field);
const char* field_name(int field);

struct ChannelDef { int b[4]; };           // sink B1 B2, source B3 B4
const std::vector<ChannelDef>& channel_table();

// One stored block type: FB_T(alpha; y0, y1, y2) = sum_terms c * N^pat_alpha(y_a0, y_a1, y_a2)
struct TypeTerm { int pat; int a[3]; double c; };
struct BlockType {
  std::vector<TypeTerm> terms;
  int pack_p = -1, pack_q = -1, pack_r = -1;  // packed pair (p, q), third position r
  int pack_sym = 0;                           // +1 symmetric, -1 antisymmetric, 0 none
  int ncell = 0, cell_off = 0;
  std::vector<int> cells;                     // cell -> y0 + 12*y1 + 144*y2
};

// pad = index of the term's channel inside its slab group
struct TermHdr { int ch, K, shape, n1, n2, off1, off2, pad; };

// Channels that read the same two stored block types (B1's at q, B2's at -q)
// form a group; one CTA of the momentum-slab contraction handles one
// (q, group).  Its work is split into items (term, first shared index of a
// 32-wide chunk), assigned to NBS_SLAB_WARPS warps with balanced cost.
#define NBS_SLAB_WARPS 4
struct GroupHdr {
  int base1, ncell1, base2, ncell2;   // cell ranges of the two types
  int ch_off, nch;                    // into Plan::group_ch (request-order channel indices)
  int item_off;                       // into Plan::items (pairs)
  int nslot;                          // partial-sum slots of all warps
  int warp_off[NBS_SLAB_WARPS + 1];   // item ranges per warp, relative to item_off
  int out_base[NBS_SLAB_WARPS + 1];   // first partial-sum slot of each warp
  int cfirst[NBS_SLAB_WARPS];         // first group channel each warp touches
  int pad[2];
};

// Persistent slab contraction: the channels of a group are split into chunks
// whose gather tables, compressed to 16 bits per entry (cell - type base in
// bits 0..9, sign in bit 10, coefficient code in bits 11..15), fit in shared
// memory; a CTA keeps one chunk's table and sweeps a block of momenta.
#define NBS_CHUNK_WARPS 8
#define NBS_CHUNK_ENTRIES 45056
#define NBS_MAX_COEF_CODES 32
struct ChunkHdr {
  int base1, ncell1, base2, ncell2;   // the group's two stored types
  int ch_off, nch;                    // into Plan::group_ch
  int tab_off, tab_len;               // 16-bit entries, into Plan::chunk_tab
  int item_off, nslot;                // into Plan::chunk_items (pairs)
  int warp_off[NBS_CHUNK_WARPS + 1];
  int out_base[NBS_CHUNK_WARPS + 1];
  int cfirst[NBS_CHUNK_WARPS];
  int ch_local0;                      // group-local index of the chunk's first channel
  int pad[3];
};

// The same chunks split over NBS_QUAD_WARPS warps for the quad-lane kernels
// (four lanes per shared index, eight indices per warp step).  Their tables
// hold the terms of a channel that share one fixed form as one run (the
// members' lists back to back, each member still addressable by its own table
// offsets), and the chunk's 8-index steps are cut into NBS_QUAD_WARPS
// contiguous ranges of about equal measured cost.  Warp w walks its range as
// the runs Plan::quad_segs[seg_base[w] .. seg_base[w + 1]) and adds its
// partial sums into slots out_base[w] + local - cfirst[w].
#define NBS_QUAD_WARPS 16
struct QuadChunkHdr {
  int base1, ncell1, base2, ncell2;
  int ch_off, nch;
  int tab_off, tab_len;
  int nslot, ch_local0;
  int out_base[NBS_QUAD_WARPS + 1];
  int cfirst[NBS_QUAD_WARPS];
  int seg_base[NBS_QUAD_WARPS + 1];
  int pad[4];  // 64 ints
};

// One run of consecutive 8-index steps inside a warp's range: shared indices
// [kbeg, kend) (kbeg a multiple of 8) of one table run, the table offsets of
// its two gather lists inside the chunk table (t1 for the lanes' own spin,
// t2 for the rows they exchange), their lengths n1, n2, the chunk-local
// channel and the form: bits 0..2 = 0..3 shape with run-time lengths, 4..7
// the fixed forms (shape 0, n 8/2), (1, 2/2), (2, 2/2), (3, 2/8); bit 3 set =
// sides exchanged (B2's list first: the run computes the transpose in
// alpha1, alpha2 of a shape-0 or shape-2 term as a shape-3 or shape-1 one).
// Only shapes 1 and 3 (forms 1, 3, 5, 7) occur.
struct QuadSeg { int form, t1, t2, kbeg, kend, local, n1, n2; };

// Two-phase contraction over distinct effective-block rows (kernels_rows.cu).
// A row of an effective block -- one shared index xi~ and one held source
// spin of one side, i.e. a sum of stored cells with coefficients -- is kept up
// to a scale: its coefficients divided by the magnitude m of its term side are
// +-1 or +-2, and its sign is fixed by its first entry.  Over all channels the
// rows depend only on the stored type they sum (and not on the channel or the
// side), a few hundred per type: phase A (Eq. (4.2)) builds every row of every
// type once per momentum, for all four sink spins, into a momentum-major array
// (its own kernel); phase B forms the product of Eq. (4.3) per chunk (whole
// channels of one slab group, i.e. one pair of stored types) from the rows of
// type1 at q and type2 at -q: record (xi~, s) names the row of B1 and of B2
// for output source-spin pair s and a scale (a code into Plan::row_scales):
// the sum of m1 m2 sign1 sign2 over the channel's products that name these two
// rows for this s.  Lane 8 g + kq of a warp takes record (step, g, kq): a
// warp step covers eight records in each of four lane groups, and a group's
// records are for one s (the step's group map), so that the four lists of a
// channel, of unequal length, share the steps.
#define NBS_ROW_WARPS 12            // consumer warps of the product kernel (record ranges)
#define NBS_ROW_HELPERS 4           // its helper warps (row copies, slot sums)
#define NBS_ROW_STAGES 3            // momenta of rows in flight per block
#define NBS_ROW_MAX_ROWS 4095       // row slots per type (12-bit row index in a record)
#define NBS_ROW_SCALES 64           // scale codes (code 63 = 0)
#define NBS_ROW_SMEM_LIMIT 232448   // shared memory per block the tables are cut for (GB300 opt-in)
// Rows of one stored type: per momentum they occupy 16-byte units
// [2 roff, 2 roff + 2 nrow) of the momentum's block of 2 row_nr units: sink
// spins 0, 1 of row r at 2 roff + r, spins 2, 3 at 2 roff + nrow + r.
struct RowTypeHdr {
  int base, ncell;                   // the stored type's cells
  int roff, nrow;                    // first row (a multiple of 8) and rows (a multiple of 8, padding rows empty)
  int pad[4];
};
struct RowChunkHdr {
  int type1, type2;                  // row types of B1 (at q) and of B2 (at -q)
  int roff1, nrow1, roff2, nrow2;    // their first rows and row counts
  int rec_off, nstep;                // 32 records (uint32) per step into Plan::row_rec
  int ch_off, nch;                   // chunk channels into Plan::row_ch (request-order indices)
  int nslot, seg_off, smem;          // per-warp partial-sum slots; segments into Plan::row_segs; bytes
  int pad0;
  int seg_base[NBS_ROW_WARPS + 1];   // warp w walks segments seg_base[w] .. seg_base[w + 1] (relative)
  int out_base[NBS_ROW_WARPS + 1];   // its slots start at out_base[w] (chunk-local channel - cfirst[w])
  int cfirst[NBS_ROW_WARPS];
  int pad[96 - 16 - 3 * NBS_ROW_WARPS];  // 96 ints
};
// Steps [sbeg, send) of chunk-local channel `local` (one flush at the end);
// lane group g (lanes 8 g + kq) holds records of output pair s = (map >> 2 g) & 3;
// bits 8 + 2 g: the group's turn among the groups of its s, bits 16..18: the turns.
struct RowSeg { int sbeg, send, local, map; };

struct Plan {
  std::vector<int> channels;                  // built-in ids, in request order
  std::vector<BlockType> types;
  int ncells = 0;
  std::vector<TermHdr> terms;
  std::vector<int> ent1_cell, ent2_cell;
  std::vector<double> ent1_coef, ent2_coef;
  std::vector<int> ch_term_begin;             // size nch + 1
  int nflav = 2;                              // propagators: 2 (l = u = d, s) or 3 (u, d, s)
  std::vector<int> ch_nl;                     // light quarks of the sink pair
  std::vector<int> ch_fl;                     // per channel: quarks of each propagator (3 ints)
  std::vector<GroupHdr> groups;
  std::vector<int> group_ch;
  std::vector<int> items;                     // pairs (term, k0)
  bool chunks_ok = false;                     // every channel fits one chunk, <= 32 coefficient codes
  std::vector<ChunkHdr> chunks;
  std::vector<unsigned short> chunk_tab;
  std::vector<int> chunk_items;               // pairs (term, k0)
  std::vector<int> term_tab_off;              // per term: side-1, side-2 offsets inside its chunk's table
  std::vector<double> coef_codes;             // |coefficient| of each code
  std::vector<QuadChunkHdr> quad_chunks;      // one per chunk (valid when chunks_ok)
  std::vector<QuadSeg> quad_segs;             // per-warp term runs of every quad chunk
  int max_quad_segs = 0;                      // most segments of one chunk
  bool rows_ok = false;                       // every chunk of the two-phase tables fits shared memory
  std::vector<RowTypeHdr> row_types;
  std::vector<unsigned> row_desc;             // per row (all types): entry offset (bits 0..23) | count << 24 | type << 29
  std::vector<unsigned short> row_ent;        // cell of the type (bits 0..11) | coefficient code (bits 12..13: +1 -1 +2 -2)
  int row_nr = 0;                             // rows per momentum (all types)
  std::vector<RowChunkHdr> row_chunks;
  std::vector<unsigned> row_rec;              // B1 row (bits 0..11) | B2 row << 12 | scale code << 24
  std::vector<int> row_ch;
  std::vector<RowSeg> row_segs;
  std::vector<double> row_scales;             // NBS_ROW_SCALES signed scales, code 63 = 0
  int row_smem = 0;                           // the largest chunk's shared memory (bytes)
  std::string row_why;                        // why rows_ok is false
  // flops of the contraction per q (complex multiply-adds), for rooflines
  double cmac_per_q = 0, gathers_per_q = 0;
};

// Source spin blocks: channel id c + n * k (n = built-in channels, k < 4)
// projects the source spins onto alpha3 in {2 (k & 1), 2 (k & 1) + 1} and
// alpha4 in {2 (k >> 1), 2 (k >> 1) + 1}; k = 0 is the upper components.
#define NBS_SPIN_BLOCKS 4

// Compile the tables for the given channel ids.  Returns "" or an error text.
std::string compile_plan(const std::vector<int>& channel_ids, Plan& out, int nflav = 2);

// Two-phase contraction tables (plan_rows.cpp); smem_limit: bytes per block.
void build_row_chunks(Plan& plan, int smem_limit);
// Shared memory of one chunk of the two-phase contraction (kernels_rows.cu layout).
size_t row_chunk_smem(int nrow1, int nrow2, int nslot, int nseg, int nch);

// Set the text that nbs_last_error(NULL) returns on this thread.
void set_global_error(const std::string& msg);

}  // namespace nbs
