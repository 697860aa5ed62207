// Internal declarations shared by the kernels (qf_kernels.cu) and the host
// planner / C ABI (qf_api.cu).  Nothing here is exported.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "qf.h"

namespace qf {

// Largest tile / block shapes handled by the fused kernels.
constexpr int kTileMaxRot = 32;   // rotations fused into one shared-memory tile pass
constexpr int kTileMaxHiBits = 9; // tile bits above the contiguous low run
constexpr int kSparseMaxRows = 8; // active rows of a sparse composite block
constexpr int kSparseMaxCls = 4;  // sign classes (2 distinct outside Z masks)
constexpr int kSparseMaxSupp = 8; // support qubits of a sparse composite block
constexpr int kChunkTerms = 4;    // Pauli terms per sign-pattern lookup table

// Rotation coefficient forms.  A rotation exp(-i th P) = c I - i s P is applied
// as out = A u + B w(v) where w(v) is the quarter-turn/sign image of the
// partner amplitude.  FORM_AB uses both coefficients (A = c*scale, B =
// s*scale); FORM_A1 has A = 1, B = tan(th) (the state keeps a factor cos(th)
// aside); FORM_B1 has A = cot(th), B = 1 (the state keeps sin(th) aside).
enum { FORM_AB = 0, FORM_A1 = 1, FORM_B1 = 2 };

struct RotArgs {
  uint64_t x, z;
  int h;     // highest set bit of x (pair pivot), -1 when x == 0
  int y;     // popc(x & z)
  int form;
  int pad;
  double A, B;
};

struct TileRot {
  uint32_t xl, zl;   // x and the in-tile part of z, in tile-local bit positions
  uint64_t zout;     // part of z outside the tile bits (a per-tile sign)
  int hl;            // highest set bit of xl, -1 when xl == 0
  int y;             // popc(x & z)
  int form;
  int pad;
  double A, B;
};

struct TileArgs {
  int m;        // rotations in this pass
  int s;        // tile bits (2^s amplitudes per tile)
  int l;        // contiguous low bits 0..l-1 in the tile
  int nhi;      // s - l tile bits above the low run
  int pos[kTileMaxHiBits];  // global positions of those bits, ascending
  int sbits[kTileMaxHiBits + 16];  // all s tile bit positions, ascending
  TileRot r[kTileMaxRot];
};

struct SparseArgs {
  int u;        // support qubits (the common x mask)
  int nr;       // active rows
  int ncls;     // sign classes (1, 2 or 4)
  int nzc;      // distinct outside-Z masks (0, 1 or 2)
  int supp[kSparseMaxSupp];      // support bit positions, ascending
  uint64_t pat[kSparseMaxRows];  // global offset of each active row
  uint64_t zc[2];
  double2 M[kSparseMaxCls][kSparseMaxRows][kSparseMaxRows];  // composite minus identity (or its inverse's)
  double2 Q[kSparseMaxCls][kSparseMaxRows][kSparseMaxRows];  // generator sum_k coeff_k P_k
};

// One X-mask group of Pauli terms for the expectation and H|psi> kernels.
struct ExpGroup {
  uint64_t x;
  int h;        // highest set bit of x, -1 for the diagonal (x = 0) group
  int nchunk;
  int chunk0;   // first chunk index
  int flags;    // bit0: has even-y terms, bit1: has odd-y terms, bit2: a single term
};

struct ExpChunk {
  uint64_t z[kChunkTerms];
  double2 tab[1 << kChunkTerms];  // (real-part weight, imaginary-part weight) per sign pattern
  float2 ftab[1 << kChunkTerms];  // the same weights in FP32 (complex64 states)
};
// A chunk's masks and real-part weights packed for n <= 32: the masks and the
// first 14 weights share one 128-byte line (one chunk per 256 bytes).
struct __align__(256) RealChunk {
  uint32_t z[kChunkTerms];
  double t[1 << kChunkTerms];
  float tf[1 << kChunkTerms];  // the same weights in FP32 (complex64 states)
};

// H|psi> plan (tiled): groups sorted by X mask form classes of equal high part
// x >> tb (tb = tile bits); a class reads one partner tile per output tile.
constexpr int kWideTerms = 8;  // terms per H|psi> sign-pattern table
constexpr int kClassTb0 = 10;  // class tables exist for tile bits 10, 11, 12
constexpr int kClassTbN = 3;
struct HClass {
  uint64_t xh;  // x >> tb
  int g0, g1;   // group range [g0, g1)
};
struct HGroup {
  uint64_t x;
  int chunk0, nchunk;
  int odd;      // some term has an odd number of Y letters (complex D)
  int pad;
};
struct WChunk {
  uint64_t z[kWideTerms];
  double2 tab[1 << kWideTerms];  // D = sum_t c_t i^{y_t} s_t: (real, imaginary) per sign pattern
};
struct WChunkF {
  uint64_t z[kWideTerms];
  float2 tab[1 << kWideTerms];
};

// Double-single H|psi> table for tiles of 2^12 amplitudes (thread t owns
// c = t + 256 k, k < 16): everything about the sign pattern that does not depend
// on the tile is precomputed here.
struct WChunkS {
  uint64_t zh[kWideTerms];   // z >> 12: the tile-index part of each term's z
  uint8_t nl[16], nh[16];    // pattern bits from the low / high nibble of (thread ^ x)
  uint8_t kx[16];            // pattern bits from element k's bits 8..11, for k ^ (x >> 8)
  float2 tab[1 << kWideTerms];  // real D split as (hi, lo) floats: D = hi + lo to ~2^-48
};

// Sector-restricted kernels (qf_sector.cu): states with fixed numbers of
// occupied even (alpha) and odd (beta) qubits.
constexpr int kSecMaxPos = 17;  // positions per parity (34 qubits)
struct SecBlk {                 // one two-row excitation block
  uint64_t pat[2];              // global offsets of the two active support patterns
  uint64_t zc[2];               // outside-Z class masks
  int nzc, ne, no, ke, ko;      // outside even/odd positions and electrons to place there
  uint32_t cnt_e, cnt_o;        // C(ne, ke), C(no, ko)
  uint8_t epos[kSecMaxPos], opos[kSecMaxPos];
  double m[kSparseMaxCls][2][2];  // composite minus identity (real), per sign class
  double q[kSparseMaxCls][2][2];  // Qi with generator Q = i Qi (reverse sweep)
};
struct SecSpace {               // all determinants of one sector
  uint32_t cnt_e, cnt_o;
  int ne, no, ke, ko;
  uint8_t epos[kSecMaxPos], opos[kSecMaxPos];
};
struct SecGroup {               // X group with its even/odd flip counts
  uint64_t x;
  int xe, xo, chunk0, nchunk;
  uint32_t xa, xb;              // x in per-spin local form (even / odd bits)
};
// Part-local sweeps.  A run is a stretch of consecutive excitation blocks whose
// supports avoid a set G of spin orbitals; the rest, U, is what the run acts
// on.  Every block of the run maps a sector member onto one with the same
// occupation of G, so the sector splits into independent parts (one per
// occupation pattern of G), and each part can take the whole run in shared
// memory, with no grid-wide synchronisation between the run's blocks.
// Inside a part, members are numbered by (alpha string on U, beta string on
// U) in "run-local" coordinates: U's alpha orbitals renumbered 0..ua-1 and its
// beta orbitals 0..ub-1.
constexpr int kRunMaxBlocks = 256;  // blocks per run (bounds one launch's length)
struct RunBlk {                     // one excitation block inside its run
  uint8_t epos[kSecMaxPos], opos[kSecMaxPos];  // run-local U orbitals outside the support
  int ne, no;                       // their counts
  int e0, o0;                       // alpha / beta electrons of the active patterns
  int nzc;
  int np;                           // parts of the run (overlap partials to reduce)
  uint32_t pu[2][2];                // pattern i on U (run-local), [i][0] alpha, [i][1] beta
  uint32_t zu[2][2];                // class mask j on U (run-local)
  uint32_t zg[2][2];                // class mask j on G (spin-local: orbital index)
  // Offsets into the run strings table (launch_sector_runs' strs) of this block's
  // outside alpha / beta strings: every subset of epos (opos), as run-local masks,
  // grouped by size k (group k starts after the C(ne, k') subsets of each k' < k),
  // each group in colex order; kNoStrings when there is no table.
  uint32_t lsa, lsb;
  double m[kSparseMaxCls][2][2];    // composite minus identity (real), per sign class
  double q[kSparseMaxCls][2][2];    // Qi with generator Q = i Qi (reverse)
  float mf[kSparseMaxCls][2][2];    // m rounded to FP32 (complex64 sweeps)
  float qf[kSparseMaxCls];          // q[c][0][1] rounded to FP32 (complex64 overlaps)
  float2 md[kSparseMaxCls][2][2];   // m as double-single (hi, lo) pairs (complex128, QF_HPSI_DS)
  float2 qd[kSparseMaxCls];         // q[c][0][1] as (hi, lo)
};
// (hi, lo) float pair of v: hi = v rounded to FP32, lo = the rest rounded.
inline float2 ds_split(double v) {
  const float hi = (float)v;
  float2 r;
  r.x = hi;
  r.y = (float)(v - (double)hi);
  return r;
}
// Fills a run block's FP32 and double-single coefficients from its FP64 ones.
inline void runblk_f32(RunBlk& B) {
  for (int c = 0; c < kSparseMaxCls; ++c) {
    for (int i = 0; i < 2; ++i)
      for (int j = 0; j < 2; ++j) {
        B.mf[c][i][j] = (float)B.m[c][i][j];
        B.md[c][i][j] = ds_split(B.m[c][i][j]);
      }
    B.qf[c] = (float)B.q[c][0][1];
    B.qd[c] = ds_split(B.q[c][0][1]);
  }
}
constexpr uint32_t kNoStrings = 0xFFFFFFFFu;
constexpr int kRunMaxOrb = 16;      // U orbitals per spin (run-local strings fit 16 bits)
struct RunPart {                    // one occupation pattern of G
  uint32_t ga, gb;                  // occupied G orbitals (spin-local masks)
  int ka, kb;                       // electrons left for U's alpha / beta orbitals
  uint32_t cnta, cntb;              // C(ua, ka), C(ub, kb): size = cnta * cntb
  uint64_t logbase;                 // first forward-log item of this part (its blocks' items follow in order)
  // Item map of the part's class (the run's parts with the same ka, kb share every
  // block's item geometry): one word per item in sweep order, laid out like the
  // log, from mapbase.  maprep: this part builds its class's map.
  uint64_t mapbase;
  int maprep;
  int pad_;
};
// An item-map word: the item's two members inside the part (12 bits each) and
// the sign-class bits its U strings give (bits 24-25).
constexpr uint32_t kMapMaxPart = 4096;
struct RunInfo {
  int b0, b1;                       // blocks [b0, b1)
  int part0, nparts;                // parts [part0, part0 + nparts), largest first
  int ua, ub;
  uint8_t apos[kSecMaxPos], bpos[kSecMaxPos];  // spin-local orbital of each run-local index
  uint32_t maxsize;                 // largest part
};

// Compact sector layout: member (alpha string a, beta string b), both as local
// masks, sits at index ra[a] * cnt_o + rb[b], where ra / rb give a string's
// colex rank among the strings with the sector's electron count (2^ne / 2^no
// entries; other entries unused).  This is the ordering the sector kernels
// enumerate members in, so member number `it` sits at index `it`.
struct SecCompact {
  const uint16_t* ra;
  const uint16_t* rb;
  uint32_t cnt_o;
};
// Groups of at most four flipped qubits, looked up by the spin orbitals they
// flip, in local indices of each parity (alpha = even qubit 2i -> i, beta = odd
// qubit 2i+1 -> i).  An entry is the group's first chunk | its chunk count << 24,
// or -1 where no group exists (groups whose chunks do not fit that code are
// listed with the large groups instead).
//   sa[i * ne + a], sb[j * no + b]                      singles
//   aa[pr(i, j) * C(ne, 2) + pr(a, b)], bb likewise     same-spin doubles, i < j, a < b
//   ab[((i * ne + a) * no + j) * no + b]                opposite-spin doubles
// with pr(i, j) = i + j (j - 1) / 2.
struct SecRank {
  const int* sa;
  const int* sb;
  const int* aa;
  const int* bb;
  const int* ab;
  int diag;                     // the x = 0 group's code, or -1
  int ne, no;
  // Real-part H|psi> weights in fixed point: itab[16 c + pat] = round(tab.x * 2^e)
  // of chunk c, inv_fix = 2^-e.  Groups of several chunks sum them exactly in
  // integer arithmetic.
  const long long* itab;
  double inv_fix;
  const RealChunk* rch;         // the chunks as RealChunk (n <= 32), else NULL
};

// Direct tables of a real molecular-type Hamiltonian on a sector (n <= 32),
// for the compact-layout H|psi>.  For a member c and a group with support S
// (the qubits its strings flip), PP_c(q) is the parity of c's occupied qubits
// below q.  When every string of the group has the Jordan-Wigner chains of S as
// its Z letters off S -- the open intervals between the 1st and 2nd and between
// the 3rd and 4th support qubits -- the group's weight on the pair (c, c ^ x) is
//     D(c) = (-1)^{xor over q in S of PP_c(q)} * W,
// with W fixed by which support qubits c occupies (the flip direction).  Single
// flips may also carry one number-operator Z_r: W = A + sum over c's occupied
// qubits r outside S of B[r].  The x = 0 group is a sum of Z strings of weight
// at most two: K + sum over occupied r of U[r] + sum over occupied r < s of
// V[r][s].  A, B, K, U, V are 64-bit fixed point (value * 2^e, inv_fix = 2^-e),
// so their sums are exact.  Local orbital q is qubit 2q (alpha) or 2q + 1 (beta).
struct SecDirect {
  int n, ne, no;               // qubits, alpha orbitals, beta orbitals
  const double* wab;           // [((o * ne + v) * no + o2) * no + v2]: c occupies alpha o, beta o2
  const double* waa;           // [pr(o1, o2) * C(ne, 2) + pr(v1, v2)]: c occupies o1 < o2, not v1 < v2
  const double* wbb;           // likewise for beta (C(no, 2))
  const float* fab;            // FP32 copies (complex64)
  const float* faa;
  const float* fbb;
  const float2* dab;           // double-single copies (hi, lo) (complex128, QF_HPSI_DS)
  const float2* daa;
  const float2* dbb;
  const long long* s1a;        // alpha single o -> v: A at [(o * ne + v) * (n + 1)], B[r] at + 1 + r
  const long long* s1b;        // beta single likewise ((o * no + v) * (n + 1))
  const long long* dg;         // K, then U[r] at 1 + r, then V[r][s] at 1 + n + r * n + s (r < s)
  double inv_fix;
};

// Kernel launchers (qf_kernels.cu).  All return cudaGetLastError() after launch.
cudaError_t launch_zero_and_set(void* psi, int n, qf_dtype dt, uint64_t det, cudaStream_t s);
// count amplitudes set to the unit vector e_idx.
cudaError_t launch_zero_and_set_count(void* psi, uint64_t count, qf_dtype dt, uint64_t idx, cudaStream_t s);
// out[2k], out[2k + 1] = (re, im) of src[idx[k]] (zeros where idx[k] < 0); packed: a
// real value kept in the imaginary slot.  ds (QF_C128, packed): that slot holds a
// double-single (hi, lo) float pair (launch_sector_runs' dss layout).
cudaError_t launch_gather(const void* src, qf_dtype dt, const int64_t* idx, int count, bool packed, bool ds,
                          double* out,
                          cudaStream_t s);
cudaError_t launch_scale(void* psi, int n, qf_dtype dt, double scale, cudaStream_t s);
cudaError_t launch_rot(void* psi, int n, qf_dtype dt, const RotArgs& a, cudaStream_t s);
cudaError_t launch_tile(void* psi, int n, qf_dtype dt, const TileArgs& a, cudaStream_t s);
// realst: the state is real (every imaginary part exactly zero) and M is real.
cudaError_t launch_sparse(void* psi, int n, qf_dtype dt, const SparseArgs& a, bool realst, cudaStream_t s);
bool sparse_m_real(const SparseArgs& a);
bool sparse_q_imag(const SparseArgs& a);
// <psi|H|psi> for the grouped plan; writes the sum into out[0] (device).
cudaError_t launch_expect(const void* psi, int n, qf_dtype dt, const ExpGroup* groups, int ngroups,
                          const ExpChunk* chunks, double* partials, unsigned* counter, double* out,
                          int nblocks, cudaStream_t s);
// lam = H psi, out[0] = Re <psi|lam>, out[1] = <psi|psi>; partials holds 2 * nblocks doubles.
cudaError_t launch_hpsi(const void* psi, void* lam, int n, qf_dtype dt, const ExpGroup* groups, int ngroups,
                        const ExpChunk* chunks, double* partials, unsigned* counter, double* out, int nblocks,
                        cudaStream_t s);
// Tiled H|psi> (n >= 8): same outputs as launch_hpsi.  tb = tile bits; chunks is a
// WChunk array (QF_C128) or a WChunkF array (QF_C64).
cudaError_t launch_hpsi_tiled(const void* psi, void* lam, int n, qf_dtype dt, int tb, bool realst,
                              const HClass* classes, int nclasses, const HGroup* groups, const void* chunks,
                              double* partials, unsigned* counter, double* out, int nblocks, cudaStream_t s);
// Tiled H|psi> for a real complex128 state and real D with double-single
// multiply-adds on the FP32 pipe (same outputs as launch_hpsi_tiled).
// split: a scratch array of 2^n float2 receiving (hi, lo) of each real part.
cudaError_t launch_hpsi_ds(const void* psi, void* lam, void* split, int n, const HClass* classes, int nclasses,
                           const HGroup* groups, const WChunkS* chunks, double* partials, unsigned* counter,
                           double* out, int nblocks, cudaStream_t s);
// Reverse step: out[0] = Im <lam|P|psi> (stored units), then psi, lam <- exp(+i th P).
cudaError_t launch_adj_rot(void* psi, void* lam, int n, qf_dtype dt, const RotArgs& a, double* partials,
                           unsigned* counter, double* out, int nblocks, cudaStream_t s);
// Reverse step over a sparse block: out[0] = Im <lam|Q|psi>, then psi, lam <- M psi, M lam
// (SparseArgs.M holds M - I for the block's inverse M).
cudaError_t launch_adj_sparse(void* psi, void* lam, int n, qf_dtype dt, const SparseArgs& a, bool realst,
                              double* partials, unsigned* counter, double* out, int nblocks, cudaStream_t s);

// Forward sector sweep over nblk blocks in one cooperative launch, full
// layout.  bar: 3 device words.  grid from sector_sweep_grid (typical_items:
// items of a typical block).
int sector_sweep_grid(uint64_t typical_items);
cudaError_t launch_sector_sweep(void* psi, qf_dtype dt, bool realst, const SecBlk* blks, int nblk, unsigned* bar,
                                int grid, cudaStream_t s);
// Part-local sweep of all runs over a compact-layout state (forward: runs and
// blocks in order, psi real; reverse: from the last, psi real and lam real
// packed in psi's imaginary slots when realst, else separate complex states).
// Reverse: out[b] = Im <lam|Q_b|psi> of block b, via partial[b * pmax + part].
// log (optional; realst only): the forward writes each item's rotated psi pair
// there (RunPart::logbase) and the reverse reads psi back from it instead of
// un-rotating psi; both sweeps of one evaluation must use the same log.
// strs: the blocks' outside strings (RunBlk::lsa / lsb), or NULL to unrank them.
// map: the plan's item maps (RunPart::mapbase), used by the forward and by the
// logged reverse, or NULL.  ds: a complex128 forward and logged reverse with maps
// run in double-single arithmetic (members and log as hi + lo float pairs, about
// 48 bits; RunBlk::md / qd); both sweeps of one evaluation must agree on it.
// dss (with ds only): the compact state itself is kept in double-single form, each
// member's slots holding (psi hi, psi lo, lam hi, lam lo) floats in place of
// (psi, lam) doubles, so that no sweep converts between the two.
// runs is a host array; parts and blks are device arrays.  Returns an error
// when a part does not fit in shared memory.
cudaError_t launch_sector_runs(void* psi, void* lam, qf_dtype dt, bool adj, bool realst, const RunInfo* runs,
                               int nruns, const RunPart* parts, const RunBlk* blks, int nblk, double* partial,
                               int pmax, double* out, const SecCompact& cm, void* log, const uint16_t* strs,
                               const uint32_t* map, bool ds, bool dss, cudaStream_t s);
// Overlaps only: out[b] = Im <lam|Q_b|psi> of every block b on the same compact
// state (psi real parts, lam real parts in psi's imaginary slots); nothing is
// rotated.  Same descriptors as launch_sector_runs.
cudaError_t launch_sector_overlaps(void* psi, qf_dtype dt, const RunInfo* runs, int nruns, const RunPart* parts,
                                  const RunBlk* blks, int nblk, double* partial, int pmax, double* out,
                                  const SecCompact& cm, const uint16_t* strs, cudaStream_t s);
// Builds the item maps (RunPart::mapbase) of every run's classes from the forward
// blocks; map holds the plan's map words.
cudaError_t launch_run_itemmaps(const RunInfo* runs, int nruns, const RunPart* parts, const RunBlk* blks,
                                const SecCompact& cm, const uint16_t* strs, uint32_t* map, cudaStream_t s);
// Largest part (members) launch_sector_runs accepts for this dtype, direction and log use.
uint32_t sector_run_capacity(qf_dtype dt, bool adj, bool realst, bool logged);
// With cm.ra != NULL psi and lam are in the compact layout.  nblocks: the
// most CTAs the reduction may use (partials holds 2 * nblocks doubles).
// lambda = H psi on the compact layout of a real state through the direct tables
// (lambda packed into psi's imaginary slots); out[0] = <psi|lambda>,
// out[1] = <psi|psi>, partials holds 2 * nblocks doubles.  split: for a
// QF_C128 state, scratch of one float2 per member that turns on double-single
// pair products (QF_HPSI_DS); NULL keeps them in FP64.  dss (with split): the
// state is in the sweeps' double-single layout (launch_sector_runs); psid,
// scratch of one double per member, receives psi, and lambda is written as a
// (hi, lo) float pair.
cudaError_t launch_sector_hpsi_direct(void* cpsi, qf_dtype dt, const SecSpace& sp, const SecDirect& d,
                                      const SecCompact& cm, double* partials, unsigned* counter, double* out,
                                      int nblocks, float2* split, double* psid, bool dss, cudaStream_t s);
cudaError_t launch_sector_hpsi(const void* psi, void* lam, qf_dtype dt, bool realst, const SecSpace& sp,
                               const SecRank& rk, const SecGroup* large, int nlarge,
                               const ExpChunk* chunks, double* partials, unsigned* counter, double* out,
                               int nblocks, const SecCompact& cm, cudaStream_t s);

// Energy and gradient of several parameter sets of one small system in one
// launch, one CTA per request, the request's compact sector state (psi and
// lambda, real) held in shared memory for the whole evaluation: the forward
// blocks, lambda = H psi through the direct tables with <psi|H|psi> and
// <psi|psi>, then the reverse blocks with their gradient overlaps.
constexpr int kSmallCoef = 36;  // per request and block: forward m[4][2][2], inverse m[4][2][2], q01[4]
struct SmallEval {
  const SecBlk* blks;  // the forward blocks' geometry (pat, zc, nzc, outside positions and counts)
  int nblk;
  const void* coef;  // per request, nblk records of kSmallCoef values of the state's real type
  SecDirect d;       // the Hamiltonian's direct tables
  uint32_t cnt_e, cnt_o;
  int ke, ko;        // the sector's alpha / beta electrons
  const uint16_t* ra;
  const uint16_t* rb;  // colex rank tables of the compact layout
  uint32_t c0;         // compact index of the reference determinant
  double* out;         // per request: the nblk block overlaps, then <psi|H|psi> and <psi|psi>
};
// Dynamic shared memory of one request's CTA (0 when it exceeds the limit).
size_t small_eval_smem(qf_dtype dt, uint32_t members, int ko, int no);
cudaError_t launch_small_eval(const SmallEval& a, qf_dtype dt, int n_req, cudaStream_t s);

// Bounded-wait self-test: words (3 device words, zeroed) -- waits on words[1]
// for limit_s seconds, then raises words[2].
cudaError_t launch_wait_selftest(unsigned* words, double limit_s, cudaStream_t s);

int reduce_blocks(int n, qf_dtype dt);  // grid size used by the reducing kernels
int prof_pre(unsigned kind, cudaStream_t s);  // kernel timing hooks (see qf_profile_begin)
void prof_post(int slot, cudaStream_t s);
void count_launch();
int profile_begin(unsigned mask);
cudaError_t profile_read(unsigned mask, uint64_t* launches, double* total_ms);
void profile_end();
void set_last_error(const std::string& msg);  // message returned by qf_last_error (this thread)

}  // namespace qf
