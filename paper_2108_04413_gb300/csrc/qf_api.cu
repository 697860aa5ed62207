// Host side of libqf: the C ABI declared in include/qf.h, the rotation planner
// (sparse composites, shared-memory tile fusion, deferred scale) and the
// X-mask grouping of Pauli sums.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <atomic>
#include <cmath>
#include <complex>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "qf_internal.h"
#include "qf_pool.h"

using cplx = std::complex<double>;

namespace {

thread_local std::string t_err;
thread_local uint64_t t_h2d = 0, t_d2h = 0;  // bytes this thread's calls copied each way

cudaError_t h2d(void* dst, const void* src, size_t bytes, cudaStream_t s) {
  t_h2d += bytes;
  return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, s);
}

cudaError_t d2h(void* dst, const void* src, size_t bytes, cudaStream_t s) {
  t_d2h += bytes;
  return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, s);
}

qf_status fail(qf_status s, const std::string& msg) {
  t_err = msg;
  return s;
}

#define QF_CUDA(expr)                                                                              \
  do {                                                                                             \
    cudaError_t e_ = (expr);                                                                       \
    if (e_ != cudaSuccess) return fail(QF_ECUDA, std::string(#expr) + ": " + cudaGetErrorString(e_)); \
  } while (0)

int popc(uint64_t v) { return __builtin_popcountll(v); }
constexpr uint64_t kEvenMask = 0x5555555555555555ull;  // alpha spin orbitals (even qubits)
int hibit(uint64_t v) { return v ? 63 - __builtin_clzll(v) : -1; }

struct ExpPlan {
  qf::ExpGroup* d_groups = nullptr;
  qf::ExpChunk* d_echunks = nullptr;  // pair-form expectation weights
  qf::ExpChunk* d_hchunks = nullptr;  // H|psi> weights
  long long* d_hfix = nullptr;        // their real parts in fixed point (SecRank::itab)
  qf::RealChunk* d_hreal = nullptr;   // their masks and real parts packed (n <= 32; SecRank::rch)
  int ngroups = 0;
  int nchunks = 0;
  // tiled H|psi>: groups in X order, 8-term tables, classes for 2^10 and 2^11 tiles
  qf::HGroup* d_hgroups = nullptr;
  qf::WChunk* d_wchunks = nullptr;
  qf::WChunkF* d_wchunks_f = nullptr;
  qf::WChunkS* d_wchunks_s = nullptr;  // real D as (hi, lo) floats for double-single H|psi>
  qf::SecGroup* d_seclarge = nullptr;   // those flipping more than four qubits
  int nseclarge = 0;
  int* d_rk = nullptr;                  // group index tables by flipped spin orbitals (see SecRank)
  qf::SecRank rk{};
  qf::HClass* d_classes[qf::kClassTbN] = {};  // classes for tile bits 10, 11, 12
  int nclasses[qf::kClassTbN] = {};
  bool tiled = false;                // tiled H|psi> tables built (on first use)
  std::vector<qf_term> terms;        // the plan's terms (compared on every cache hit; tiled tables)
  bool has_odd = false;  // some term has an odd number of Y letters (imaginary phase)
  uint64_t last_use = 0; // the handle's call count at the plan's last use (least recently used goes first)
  // direct sector H|psi> tables (qf::SecDirect): 0 not tried yet, 1 built, -1 the
  // terms do not take that form (the chunk-table kernel runs instead)
  int direct = 0;
  void* d_direct = nullptr;
  qf::SecDirect dtab{};
};

void free_plan(ExpPlan& p) {
  cudaFree(p.d_groups);
  cudaFree(p.d_echunks);
  cudaFree(p.d_hchunks);
  cudaFree(p.d_hfix);
  cudaFree(p.d_hreal);
  cudaFree(p.d_hgroups);
  cudaFree(p.d_wchunks);
  cudaFree(p.d_wchunks_f);
  cudaFree(p.d_wchunks_s);
  cudaFree(p.d_seclarge);
  cudaFree(p.d_rk);
  cudaFree(p.d_direct);
  for (int v = 0; v < qf::kClassTbN; ++v) cudaFree(p.d_classes[v]);
  p = ExpPlan();
}

// Content key of a host array: four independent multiply-rotate lanes over
// 8-byte words (the tail byte-wise), then a xor-shift-multiply finish.  Used to
// recognise a term list or an ansatz seen before; a different array colliding
// has probability ~2^-64.
inline uint64_t rotl64(uint64_t v, int s) { return (v << s) | (v >> (64 - s)); }
uint64_t content_key(const void* data, size_t bytes, uint64_t seed = 0x243F6A8885A308D3ull) {
  const unsigned char* p = static_cast<const unsigned char*>(data);
  const uint64_t K1 = 0x9E3779B97F4A7C15ull, K2 = 0xC2B2AE3D27D4EB4Full;
  uint64_t h[4] = {seed, seed ^ K1, seed ^ K2, seed + bytes};
  size_t i = 0;
  for (; i + 32 <= bytes; i += 32)
    for (int l = 0; l < 4; ++l) {
      uint64_t w;
      std::memcpy(&w, p + i + 8 * l, 8);
      h[l] = rotl64(h[l] ^ (w * K2), 31) * K1;
    }
  uint64_t v = h[0] ^ rotl64(h[1], 17) ^ rotl64(h[2], 33) ^ rotl64(h[3], 49);
  for (; i < bytes; ++i) v = (v ^ p[i]) * K1;
  v ^= v >> 32;
  v *= 0xD6E8FEB86659FD93ull;
  v ^= v >> 32;
  v *= 0xD6E8FEB86659FD93ull;
  v ^= v >> 32;
  return v;
}

// Whether a cached plan's rotation list equals the caller's.
bool same_arots(const std::vector<qf_arot>& seen, const qf_arot* a, size_t n) {
  return seen.size() == n && (n == 0 || std::memcmp(seen.data(), a, n * sizeof(qf_arot)) == 0);
}

}  // namespace

void qf::set_last_error(const std::string& msg) { t_err = msg; }

// Host allocator of page-locked memory (cudaMallocHost), so that an array
// refilled and uploaded on every call goes to the device by an asynchronous DMA
// instead of a staged pageable copy.  Falls back to ordinary memory when the
// page-locked allocation fails; a 16-byte header records which one it is.
template <typename T>
struct PinnedAlloc {
  using value_type = T;
  PinnedAlloc() = default;
  template <typename U>
  PinnedAlloc(const PinnedAlloc<U>&) {}
  T* allocate(size_t n) {
    const size_t bytes = n * sizeof(T) + 16;
    void* p = nullptr;
    unsigned char tag = 1;
    if (cudaMallocHost(&p, bytes) != cudaSuccess) {
      cudaGetLastError();
      p = std::malloc(bytes);
      tag = 0;
      if (!p) throw std::bad_alloc();
    }
    static_cast<unsigned char*>(p)[0] = tag;
    return reinterpret_cast<T*>(static_cast<unsigned char*>(p) + 16);
  }
  void deallocate(T* q, size_t) {
    unsigned char* p = reinterpret_cast<unsigned char*>(q) - 16;
    if (p[0])
      cudaFreeHost(p);
    else
      std::free(p);
  }
  template <typename U>
  bool operator==(const PinnedAlloc<U>&) const { return true; }
  template <typename U>
  bool operator!=(const PinnedAlloc<U>&) const { return false; }
};

// The part-local run plan of an ansatz in one sector (see build_runs).
struct SectorRuns {
  std::vector<qf::RunInfo> runs;
  std::vector<qf::RunPart> parts;
  // forward blocks, then inverse blocks (m, q refilled and uploaded per call)
  std::vector<qf::RunBlk, PinnedAlloc<qf::RunBlk>> blks;
  int pmax = 0;
  uint64_t logitems = 0;         // (member pair, block) items of one sweep: the forward log's length
  std::vector<uint64_t> run_items;  // the items of each run (they sum to logitems)
  std::vector<uint16_t> strs;    // the blocks' outside strings (RunBlk::lsa / lsb); empty when not tabulated
  bool log_ok = true;            // every inverse block lists its two patterns in the forward order
  // item maps (RunPart::mapbase): words of all classes; map_ok when every part fits
  // a map word and the inverse blocks share the forward blocks' item geometry
  uint64_t mapwords = 0;
  bool map_ok = false;
};

struct qf_state {
  int n = 0;
  qf_dtype dt = QF_C128;
  cudaStream_t stream = nullptr;
  void* psi = nullptr;
  bool own_psi = false;
  void* lam = nullptr;
  void* split = nullptr;  // (hi, lo) float copy of psi's real parts for double-single H|psi>
  double scale = 1.0;
  // Every stored imaginary part is exactly zero.  Holds after qf_set_basis and
  // is kept by real sparse composites and by rotations with x != 0 and an odd
  // number of Y letters (their phases map real amplitudes to real ones).
  bool real = true;
  // Numbers of occupied even (alpha) and odd (beta) qubits when every nonzero
  // amplitude has them (set by qf_set_basis, kept by sector-preserving blocks);
  // -1 when unknown.
  int sec_a = -1, sec_b = -1;
  qf::SecBlk* d_secblk = nullptr;  // sector block descriptors (forward, then reverse)
  size_t secblk_cap = 0;
  double* d_sec_partial = nullptr;  // reverse-sweep overlaps per block and CTA
  size_t sec_partial_cap = 0;
  unsigned* d_bar = nullptr;        // grid barrier words
  // compact sector layout of qf_energy_grad: rank tables of sector (rank_n,
  // rank_a, rank_b) and the compact psi / lambda buffer
  uint16_t* d_rank = nullptr;
  int rank_n = -1, rank_a = -1, rank_b = -1;
  void* d_cstate = nullptr;
  size_t cstate_cap = 0;
  void* d_runblk = nullptr;  // part-local sweep descriptors (blocks, then parts)
  size_t runblk_cap = 0;
  void* d_idx = nullptr;     // residual read-out indices
  size_t idx_cap = 0;
  void* d_poolblk = nullptr; // operator-pool run descriptors (blocks, parts, strings)
  size_t poolblk_cap = 0;
  uint64_t pool_key = 0;     // the pool plan and sector whose descriptors sit in d_poolblk
  void* d_map = nullptr;     // item maps of the part-local sweeps (RunPart::mapbase)
  size_t map_cap = 0;
  uint64_t map_key = 0;      // the plan and sector whose maps sit in d_map
  void* d_log = nullptr;     // forward log of the part-local sweeps (psi pairs after each block)
  size_t log_cap = 0;
  bool log_failed = false;   // the log did not fit: later calls un-rotate psi instead
  int hpsi_mode = QF_HPSI_DS;
  // several parameter sets in one launch (qf_energy_grad_multi): the plan's block
  // geometries for one sector (small_key), per-request coefficients and results
  void* d_small = nullptr;
  size_t small_cap = 0;
  uint64_t small_key = 0;
  void* d_scoef = nullptr;
  size_t scoef_cap = 0;
  void* h_scoef = nullptr;  // page-locked
  size_t h_scoef_cap = 0;
  void* d_sout = nullptr;
  size_t sout_cap = 0;
  void* h_sout = nullptr;  // page-locked
  size_t h_sout_cap = 0;
  double* d_partials = nullptr;
  unsigned* d_counter = nullptr;
  double* d_out = nullptr;
  size_t out_cap = 0;
  double* h_out = nullptr;
  size_t h_cap = 0;
  std::unordered_map<uint64_t, ExpPlan> plans;
  // block structure of ansatz lists seen by qf_energy_grad (angles refilled per call)
  struct Blk {
    size_t i, j;
    bool sparse;
    qf::SparseArgs fwd, inv;  // filled by build_sparse (which clears them) when sparse
    Blk() {}                  // no zeroing: a plan holds thousands of ~16 KB blocks
  };
  struct AnsatzPlan {
    std::vector<qf_arot> src;  // the rotation list it was planned from (compared on every cache hit)
    uint64_t last_use = 0;
    std::vector<Blk> blocks;
    // sector run plan, built for (sec_n, sec_na, sec_nb) on first use there
    int sec_n = -1, sec_na = -1, sec_nb = -1;
    uint64_t sec_cap = 0;
    bool sec_ok = false;
    SectorRuns runs;
  };
  std::unordered_map<uint64_t, AnsatzPlan> ansatz_plans;
  uint64_t parts_key = 0;  // the ansatz plan and sector whose run parts sit in d_runblk
  // keys of the last Pauli-sum and ansatz plans used: compared first, without hashing
  uint64_t last_plan_key = 0, last_ansatz_key = 0;
  std::vector<uint64_t> run_items;  // items of each run of the last part-local sweep (launch order)
  uint64_t calls = 0;      // plan-using calls so far (the caches' clock)
  size_t elem() const { return dt == QF_C128 ? 16 : 8; }
  size_t bytes() const { return elem() << n; }
};

namespace {

constexpr int kPartials = 4096;
// Target part size (members) of the part-local sector sweeps: ~40 KB of shared
// memory per part, so several parts run on each SM.
constexpr uint64_t kRunPartTarget = 4096;
// Largest outside-string table of a run plan (uint16 entries: 64 MB).
constexpr uint64_t kStringsMax = (uint64_t)1 << 25;
// Largest forward log of the part-local sweeps a handle allocates (24 qubits,
// complex128: 2.1 GB).
constexpr size_t kLogMaxBytes = (size_t)16 << 30;
// Largest item-map table a handle allocates (words; 1 GB).
constexpr uint64_t kMapMaxWords = (uint64_t)1 << 28;
// Plans a handle keeps per cache (Pauli sums; ansatz and pool block structures).
// Past that, the least recently used are dropped (with their device tables) when
// the next plan-using call starts, so no call loses a plan it is using.
constexpr size_t kMaxPlans = 8;

void free_plan(ExpPlan& p);

// Drop the least recently used plans beyond kMaxPlans; stamps the call.
void trim_plans(qf_state* st) {
  ++st->calls;
  while (st->plans.size() > kMaxPlans) {
    auto lru = st->plans.begin();
    for (auto it = st->plans.begin(); it != st->plans.end(); ++it)
      if (it->second.last_use < lru->second.last_use) lru = it;
    free_plan(lru->second);
    st->plans.erase(lru);
  }
  while (st->ansatz_plans.size() > kMaxPlans) {
    auto lru = st->ansatz_plans.begin();
    for (auto it = st->ansatz_plans.begin(); it != st->ansatz_plans.end(); ++it)
      if (it->second.last_use < lru->second.last_use) lru = it;
    st->ansatz_plans.erase(lru);
    st->parts_key = 0;  // descriptors on the device are re-uploaded by their next user
    st->map_key = 0;
    st->pool_key = 0;
  }
}

// Bits of mask on qubits of parity par (0 even / alpha, 1 odd / beta), as local
// spin-orbital indices: qubit q -> bit q >> 1.
uint32_t local_bits(uint64_t mask, int par) {
  uint32_t out = 0;
  for (int q = par; q < 64; q += 2)
    if ((mask >> q) & 1ull) out |= 1u << (q >> 1);
  return out;
}

// Largest |log2 scale| kept aside before it is folded back into the amplitudes.
double scale_limit(qf_dtype dt) { return dt == QF_C128 ? 400.0 : 30.0; }

// Coefficients for exp(-i th P) = c I - i s P given the scale kept aside
// (amplitudes = scale * stored values); updates that scale.  The larger of
// |c| and |s| is factored out so the kernel needs one FMA per real component.
void rot_coeffs(qf_dtype dt, double* scale, double th, int* form, double* A, double* B) {
  const double c = std::cos(th), s = std::sin(th);
  if (std::fabs(std::log2(std::fabs(*scale))) > scale_limit(dt)) {
    *form = qf::FORM_AB;
    *A = c * *scale;
    *B = s * *scale;
    *scale = 1.0;
  } else if (std::fabs(c) >= std::fabs(s)) {
    *form = qf::FORM_A1;
    *A = 1.0;
    *B = s / c;
    *scale *= c;
  } else {
    *form = qf::FORM_B1;
    *A = c / s;
    *B = 1.0;
    *scale *= s;
  }
}

qf::RotArgs rot_args(qf_dtype dt, double* scale, uint64_t x, uint64_t z, double th) {
  qf::RotArgs a{};
  a.x = x;
  a.z = z;
  a.h = hibit(x);
  a.y = popc(x & z);
  rot_coeffs(dt, scale, th, &a.form, &a.A, &a.B);
  return a;
}

// A rotation keeps a real state real iff x != 0 and popc(x & z) is odd.
bool keeps_real(uint64_t x, uint64_t z) { return x != 0 && (popc(x & z) & 1); }

qf_status ensure_out(qf_state* st, size_t n) {
  if (n <= st->out_cap) return QF_OK;
  size_t cap = std::max<size_t>(n, 2 * st->out_cap);
  if (st->d_out) cudaFree(st->d_out);
  if (st->h_out) cudaFreeHost(st->h_out);
  st->d_out = nullptr;
  st->h_out = nullptr;
  st->out_cap = 0;
  if (cudaMalloc(&st->d_out, cap * sizeof(double)) != cudaSuccess) return fail(QF_ENOMEM, "cudaMalloc(out) failed");
  if (cudaMallocHost(&st->h_out, cap * sizeof(double)) != cudaSuccess)
    return fail(QF_ENOMEM, "cudaMallocHost(out) failed");
  st->out_cap = cap;
  return QF_OK;
}

// Term indices ordered by X mask, equal masks in input order (a stable sort by
// x), through (x, index) pairs: contiguous keys, no indirection per comparison.
std::vector<size_t> order_by_x(const qf_term* T, size_t nt) {
  std::vector<std::pair<uint64_t, size_t>> key(nt);
  for (size_t i = 0; i < nt; ++i) key[i] = {T[i].x, i};
  std::sort(key.begin(), key.end());
  std::vector<size_t> order(nt);
  for (size_t i = 0; i < nt; ++i) order[i] = key[i].second;
  return order;
}

qf_status validate_masks(const qf_state* st, uint64_t x, uint64_t z) {
  const uint64_t lim = (st->n >= 64) ? ~0ull : ((1ull << st->n) - 1ull);
  if ((x & ~lim) || (z & ~lim)) return fail(QF_EINVAL, "Pauli mask has a bit at or above the qubit count");
  return QF_OK;
}

// ---------------------------------------------------------------------------
// Pauli-sum plan: group by X mask, pack terms four per chunk with sign-pattern
// tables (Eq. 18 evaluated pair by pair).

qf_status get_plan(qf_state* st, const qf_term* terms, size_t nt, const ExpPlan** out) {
  auto same_terms = [&](const std::vector<qf_term>& seen) {
    return seen.size() == nt && (nt == 0 || std::memcmp(seen.data(), terms, nt * sizeof(qf_term)) == 0);
  };
  // a loop over one Hamiltonian finds its plan with one comparison, no hashing
  auto last = st->plans.find(st->last_plan_key);
  if (last != st->plans.end() && same_terms(last->second.terms)) {
    last->second.last_use = st->calls;
    *out = &last->second;
    return QF_OK;
  }
  const uint64_t key = content_key(terms, nt * sizeof(qf_term), 0x243F6A8885A308D3ull ^ (uint64_t)st->n);
  auto it = st->plans.find(key);
  if (it != st->plans.end()) {
    if (same_terms(it->second.terms)) {
      st->last_plan_key = key;
      it->second.last_use = st->calls;
      *out = &it->second;
      return QF_OK;
    }
    // another term list with the same key: the key only picks the slot, so replace it
    free_plan(it->second);
    st->plans.erase(it);
  }
  // a term list not seen before: its masks are checked once, here (a cached plan's
  // terms were checked when it was built)
  for (size_t k = 0; k < nt; ++k) {
    qf_status v = validate_masks(st, terms[k].x, terms[k].z);
    if (v != QF_OK) return v;
  }
  st->last_plan_key = key;
  // terms grouped by X mask: ascending x, each group's terms in input order
  const std::vector<size_t> order = order_by_x(terms, nt);
  std::vector<qf::ExpGroup> groups;
  std::vector<qf::ExpChunk> ech, hch;
  ech.reserve(nt);  // at most one chunk per term: the tables are built in place
  hch.reserve(nt);
  // scratch reused across groups
  std::vector<size_t> idx;
  // the group's chunks, flat: chunk c holds terms pterm[poff[c] .. poff[c + 1])
  // with coordinates pcrd (same range) over the basis pbas[boff[c] .. boff[c + 1])
  std::vector<size_t> pterm, poff, boff;
  std::vector<uint32_t> pcrd;
  std::vector<uint64_t> pbas;
  std::vector<uint64_t> B, E;
  std::vector<uint32_t> Cb, a;
  std::vector<double> addh, adde;  // a term's exact table addend (real or imaginary part) before its sign
  std::vector<char> odd;           // the addend is imaginary (odd number of Y)
  for (size_t q0 = 0; q0 < nt;) {
    size_t q1 = q0 + 1;
    while (q1 < nt && terms[order[q1]].x == terms[order[q0]].x) ++q1;
    idx.assign(order.begin() + q0, order.begin() + q1);
    q0 = q1;
    qf::ExpGroup g{};
    g.x = terms[idx[0]].x;
    g.h = hibit(g.x);
    g.chunk0 = (int)ech.size();
    g.flags = 0;
    for (size_t i : idx) g.flags |= (popc(terms[i].x & terms[i].z) & 1) ? 2 : 1;
    if (idx.size() == 1) g.flags |= 4;  // one term: its table is +-tab[0] (k_expect_tiled)
    // A chunk holds terms whose Z masks are combinations (over GF(2)) of at most
    // kChunkTerms basis masks: the table entry for the basis parities `pat` sums
    // the terms with the sign (-1)^{popc(a_t & pat)}, a_t the term's coordinates.
    // When the whole group spans at most kChunkTerms dimensions it is one chunk;
    // otherwise each chunk takes kChunkTerms terms as its own basis.
    pterm.clear();
    pcrd.clear();
    pbas.clear();
    poff.assign(1, 0);
    boff.assign(1, 0);
    {
      B.clear();  // basis (term masks)
      E.clear();  // echelon copies (pivot = highest bit, descending)
      Cb.clear(); // E[i] as a combination of B
      a.assign(idx.size(), 0u);
      bool fits = true;
      for (size_t t = 0; t < idx.size() && fits; ++t) {
        uint64_t v = terms[idx[t]].z;
        uint32_t comb = 0;
        for (size_t i = 0; i < E.size(); ++i)
          if ((v >> hibit(E[i])) & 1ull) {
            v ^= E[i];
            comb ^= Cb[i];
          }
        if (v == 0) {
          a[t] = comb;
          continue;
        }
        if ((int)B.size() == qf::kChunkTerms) {
          fits = false;
          break;
        }
        const uint32_t j = (uint32_t)B.size();
        B.push_back(terms[idx[t]].z);
        size_t pos = 0;  // keep E sorted by pivot, descending
        while (pos < E.size() && hibit(E[pos]) > hibit(v)) ++pos;
        E.insert(E.begin() + pos, v);
        Cb.insert(Cb.begin() + pos, comb ^ (1u << j));
        a[t] = 1u << j;
      }
      if (fits) {
        pterm.assign(idx.begin(), idx.end());
        pcrd.assign(a.begin(), a.end());
        pbas.assign(B.begin(), B.end());
        poff.push_back(pterm.size());
        boff.push_back(pbas.size());
      } else {
        for (size_t k = 0; k < idx.size(); k += qf::kChunkTerms) {
          const size_t cnt = std::min<size_t>(qf::kChunkTerms, idx.size() - k);
          for (size_t t = 0; t < cnt; ++t) {
            pterm.push_back(idx[k + t]);
            pcrd.push_back(1u << t);
            pbas.push_back(terms[idx[k + t]].z);
          }
          poff.push_back(pterm.size());
          boff.push_back(pbas.size());
        }
      }
    }
    const size_t nch = poff.size() - 1;
    g.nchunk = (int)nch;
    for (size_t c = 0; c < nch; ++c) {
      qf::ExpChunk& ce = ech.emplace_back();
      qf::ExpChunk& ch = hch.emplace_back();
      const size_t* cterm = pterm.data() + poff[c];
      const uint32_t* ccrd = pcrd.data() + poff[c];
      const uint64_t* cbas = pbas.data() + boff[c];
      const int nbas = (int)(boff[c + 1] - boff[c]);
      for (int t = 0; t < qf::kChunkTerms; ++t) ce.z[t] = ch.z[t] = (t < nbas) ? cbas[t] : 0ull;
      // per term: i^y c (real for even y, imaginary for odd y) and the expectation
      // weight (1 for x = 0, else 2 for the two pair members; odd y: 2 c (-1)^{(y+1)/2});
      // each is exact up to the sign the pattern gives it
      const size_t nterm = poff[c + 1] - poff[c];
      addh.resize(nterm);
      adde.resize(nterm);
      odd.resize(nterm);
      for (size_t t = 0; t < nterm; ++t) {
        const qf_term& T = terms[cterm[t]];
        const int y = popc(T.x & T.z) & 3;
        odd[t] = (char)(y & 1);
        if ((y & 1) == 0) {
          const double ph = (y == 2) ? -1.0 : 1.0;  // i^y
          addh[t] = T.coeff * ph;
          adde[t] = (g.x == 0 ? 1.0 : 2.0) * T.coeff * ph;
        } else {
          addh[t] = T.coeff * ((y == 3) ? -1.0 : 1.0);           // i^y = +-i
          adde[t] = 2.0 * T.coeff * ((y == 1) ? -1.0 : 1.0);     // 2 c (-1)^{(y+1)/2}
        }
      }
      for (int pat = 0; pat < (1 << qf::kChunkTerms); ++pat) {
        double ex = 0, ey = 0, hx = 0, hy = 0;
        for (size_t t = 0; t < nterm; ++t) {
          const bool neg = popc(ccrd[t] & (uint32_t)pat) & 1;
          const double h = neg ? -addh[t] : addh[t], e = neg ? -adde[t] : adde[t];
          if (!odd[t]) {
            hx += h;
            ex += e;
          } else {
            hy += h;
            ey += e;
          }
        }
        ce.tab[pat] = make_double2(ex, ey);
        ch.tab[pat] = make_double2(hx, hy);
        ce.ftab[pat] = make_float2((float)ex, (float)ey);
        ch.ftab[pat] = make_float2((float)hx, (float)hy);
      }
    }
    groups.push_back(g);
  }
  // fixed-point real weights for groups of several chunks: the largest |D| such a
  // group can reach, times 2^e, stays below 2^61
  double maxabs = 0.0;
  for (const qf::ExpGroup& g : groups) {
    if (g.nchunk < 2) continue;
    double m = 0.0;
    for (int c = 0; c < g.nchunk; ++c) {
      double cm = 0.0;
      for (int pat = 0; pat < (1 << qf::kChunkTerms); ++pat) cm = std::max(cm, std::fabs(hch[g.chunk0 + c].tab[pat].x));
      m += cm;
    }
    maxabs = std::max(maxabs, m);
  }
  int fix_e = 0;
  if (maxabs > 0.0) fix_e = std::min(1000, 61 - (int)std::ceil(std::log2(maxabs)));
  const double inv_fix = std::ldexp(1.0, -fix_e);
  std::vector<long long> hfix(hch.size() << qf::kChunkTerms);
  for (size_t c = 0; c < hch.size(); ++c)
    for (int pat = 0; pat < (1 << qf::kChunkTerms); ++pat)
      hfix[(c << qf::kChunkTerms) + pat] = std::llrint(std::ldexp(hch[c].tab[pat].x, fix_e));
  ExpPlan p;
  p.ngroups = (int)groups.size();
  p.nchunks = (int)ech.size();
  for (const qf::ExpGroup& g : groups)
    if (g.flags & 2) p.has_odd = true;
  // sector groups: a group flips popc(x & even) even qubits; it links two members of
  // one sector only when that count (and the odd one) is even
  std::vector<qf::SecGroup> sg;
  for (const qf::ExpGroup& g : groups) {
    const int xe = popc(g.x & kEvenMask), xo = popc(g.x & ~kEvenMask);
    if ((xe & 1) || (xo & 1)) continue;
    sg.push_back(qf::SecGroup{g.x, xe, xo, g.chunk0, g.nchunk, local_bits(g.x, 0), local_bits(g.x, 1)});
  }
  // lookup tables by flipped spin orbitals (local index i of qubit 2i or 2i+1)
  const int nq = st->n, ne = (nq + 1) / 2, no = nq / 2;
  const int pe = ne * (ne - 1) / 2, po = no * (no - 1) / 2;
  const size_t o_sa = 0, o_sb = o_sa + (size_t)ne * ne, o_aa = o_sb + (size_t)no * no,
               o_bb = o_aa + (size_t)pe * pe, o_ab = o_bb + (size_t)po * po,
               n_rk = o_ab + (size_t)ne * ne * no * no;
  std::vector<int> rkt(std::max<size_t>(1, n_rk), -1);
  std::vector<qf::SecGroup> lg;
  int diag = -1;
  auto pr = [](int i, int j) { return i + j * (j - 1) / 2; };  // i < j
  for (size_t gi = 0; gi < sg.size(); ++gi) {
    const uint64_t x = sg[gi].x;
    const int w = popc(x);
    // table entries hold the group's chunk0 | nchunk << 24; a group that does not
    // fit that code is tested one by one with the large groups
    if (sg[gi].chunk0 >= (1 << 24) || sg[gi].nchunk > 127) {
      lg.push_back(sg[gi]);
      continue;
    }
    const int code = sg[gi].chunk0 | (sg[gi].nchunk << 24);
    int ev[32], od[32], nev = 0, nod = 0;  // flipped alpha / beta orbitals (n <= 64)
    for (int q = 0; q < nq; ++q)
      if ((x >> q) & 1) {
        if (q & 1) od[nod++] = q >> 1;
        else ev[nev++] = q >> 1;
      }
    if (w == 0) {
      diag = code;
      continue;
    }
    // each flip set is recorded under every occupied/empty split that a member can present
    if (w == 2 && nev == 2) {
      rkt[o_sa + ev[0] * ne + ev[1]] = code;
      rkt[o_sa + ev[1] * ne + ev[0]] = code;
    } else if (w == 2 && nod == 2) {
      rkt[o_sb + od[0] * no + od[1]] = code;
      rkt[o_sb + od[1] * no + od[0]] = code;
    } else if (w == 4 && (nev == 4 || nod == 4)) {
      const int* v = nev == 4 ? ev : od;
      const size_t off = nev == 4 ? o_aa : o_bb;
      const int P = nev == 4 ? pe : po;
      const int pairs[3][4] = {{0, 1, 2, 3}, {0, 2, 1, 3}, {0, 3, 1, 2}};
      for (const auto& q : pairs) {
        const int r1 = pr(v[q[0]], v[q[1]]), r2 = pr(v[q[2]], v[q[3]]);
        rkt[off + (size_t)r1 * P + r2] = code;
        rkt[off + (size_t)r2 * P + r1] = code;
      }
    } else if (w == 4 && nev == 2) {
      for (int s0 = 0; s0 < 2; ++s0)
        for (int s1 = 0; s1 < 2; ++s1)
          rkt[o_ab + (((size_t)ev[s0] * ne + ev[1 - s0]) * no + od[s1]) * no + od[1 - s1]] = code;
    } else {
      lg.push_back(sg[gi]);
    }
  }
  p.nseclarge = (int)lg.size();
  if (p.ngroups > 0) {
    if (cudaMalloc(&p.d_groups, groups.size() * sizeof(qf::ExpGroup)) != cudaSuccess ||
        cudaMalloc(&p.d_echunks, ech.size() * sizeof(qf::ExpChunk)) != cudaSuccess ||
        cudaMalloc(&p.d_hchunks, hch.size() * sizeof(qf::ExpChunk)) != cudaSuccess) {
      cudaFree(p.d_groups);
      cudaFree(p.d_echunks);
      cudaFree(p.d_hchunks);
      return fail(QF_ENOMEM, "cudaMalloc(plan) failed");
    }
    QF_CUDA(h2d(p.d_groups, groups.data(), groups.size() * sizeof(qf::ExpGroup), st->stream));
    QF_CUDA(h2d(p.d_echunks, ech.data(), ech.size() * sizeof(qf::ExpChunk), st->stream));
    QF_CUDA(h2d(p.d_hchunks, hch.data(), hch.size() * sizeof(qf::ExpChunk), st->stream));
    if (cudaMalloc(&p.d_hfix, std::max<size_t>(1, hfix.size()) * sizeof(long long)) != cudaSuccess) {
      cudaGetLastError();
      p.d_hfix = nullptr;
      free_plan(p);
      return fail(QF_ENOMEM, "cudaMalloc(plan) failed");
    }
    if (!hfix.empty()) QF_CUDA(h2d(p.d_hfix, hfix.data(), hfix.size() * sizeof(long long), st->stream));
    if (st->n <= 32 && !hch.empty()) {
      std::vector<qf::RealChunk> rc(hch.size());
      for (size_t c = 0; c < hch.size(); ++c) {
        for (int t = 0; t < qf::kChunkTerms; ++t) rc[c].z[t] = (uint32_t)hch[c].z[t];
        for (int pat = 0; pat < (1 << qf::kChunkTerms); ++pat) {
          rc[c].t[pat] = hch[c].tab[pat].x;
          rc[c].tf[pat] = (float)hch[c].tab[pat].x;
        }
      }
      if (cudaMalloc(&p.d_hreal, rc.size() * sizeof(qf::RealChunk)) != cudaSuccess) {
        cudaGetLastError();
        p.d_hreal = nullptr;
        free_plan(p);
        return fail(QF_ENOMEM, "cudaMalloc(plan) failed");
      }
      QF_CUDA(h2d(p.d_hreal, rc.data(), rc.size() * sizeof(qf::RealChunk), st->stream));
    }
    if (cudaMalloc(&p.d_seclarge, std::max<size_t>(1, lg.size()) * sizeof(qf::SecGroup)) != cudaSuccess ||
        cudaMalloc(&p.d_rk, rkt.size() * sizeof(int)) != cudaSuccess) {
      cudaGetLastError();
      free_plan(p);
      return fail(QF_ENOMEM, "cudaMalloc(plan) failed");
    }
    if (!lg.empty()) QF_CUDA(h2d(p.d_seclarge, lg.data(), lg.size() * sizeof(qf::SecGroup), st->stream));
    QF_CUDA(h2d(p.d_rk, rkt.data(), rkt.size() * sizeof(int), st->stream));
    p.rk = qf::SecRank{p.d_rk + o_sa, p.d_rk + o_sb, p.d_rk + o_aa, p.d_rk + o_bb, p.d_rk + o_ab, diag, ne, no,
                       p.d_hfix, inv_fix, p.d_hreal};
    QF_CUDA(cudaStreamSynchronize(st->stream));
  }
  p.terms.assign(terms, terms + nt);
  p.last_use = st->calls;
  auto res = st->plans.emplace(key, std::move(p));
  *out = &res.first->second;
  return QF_OK;
}

// ---------------------------------------------------------------------------
// Direct sector tables (qf::SecDirect) of a real Pauli sum on n <= 32 qubits.
// Every group that can link two members of one sector must take the form the
// direct kernel evaluates: all strings with an even number of Y letters; for a
// flip set S of two or four qubits, Z letters off S equal to the Jordan-Wigner
// chains of S (open intervals between the 1st and 2nd and between the 3rd and
// 4th support qubits), a two-qubit flip may add one more Z; the x = 0 group has
// Z strings of weight at most two.  A molecular Hamiltonian (Eq. 1 through
// Eq. 15-16) takes this form.  Returns false otherwise.
struct DirectHost {
  std::vector<double> wab, waa, wbb;  // doubles' weights
  std::vector<double> s1a, s1b;       // singles' A and B (before fixed point)
  std::vector<double> dg;             // K, U, V (before fixed point)
};

bool build_direct(const std::vector<qf_term>& T, int n, DirectHost* h) {
  if (n < 2 || n > 32) return false;
  const int ne = (n + 1) / 2, no = n / 2, pe = ne * (ne - 1) / 2, po = no * (no - 1) / 2;
  h->wab.assign((size_t)ne * ne * no * no, 0.0);
  h->waa.assign((size_t)std::max(1, pe * pe), 0.0);
  h->wbb.assign((size_t)std::max(1, po * po), 0.0);
  h->s1a.assign((size_t)ne * ne * (n + 1), 0.0);
  h->s1b.assign((size_t)no * no * (n + 1), 0.0);
  h->dg.assign((size_t)1 + n + (size_t)n * n, 0.0);
  const std::vector<size_t> order = order_by_x(T.data(), T.size());
  auto pr = [](int i, int j) { return i + j * (j - 1) / 2; };  // i < j
  std::vector<double> wr(n);
  for (size_t q0 = 0; q0 < order.size();) {
    size_t q1 = q0 + 1;
    const uint64_t x = T[order[q0]].x;
    while (q1 < order.size() && T[order[q1]].x == x) ++q1;
    const int xe = popc(x & kEvenMask), xo = popc(x & ~kEvenMask);
    if ((xe & 1) || (xo & 1)) {  // never links two members of one sector
      q0 = q1;
      continue;
    }
    for (size_t k = q0; k < q1; ++k)
      if (popc(T[order[k]].x & T[order[k]].z) & 1) return false;  // imaginary weight
    if (x == 0) {
      for (size_t k = q0; k < q1; ++k) {
        const qf_term& t = T[order[k]];
        int zb[32], nz = 0;  // n <= 32
        for (int q = 0; q < n; ++q)
          if ((t.z >> q) & 1ull) zb[nz++] = q;
        if (nz > 2) return false;
        // (-1)^{c_r} = 1 - 2 c_r on occupation bits c_r
        h->dg[0] += t.coeff;
        for (int i = 0; i < nz; ++i) h->dg[1 + zb[i]] -= 2.0 * t.coeff;
        if (nz == 2) h->dg[1 + n + (size_t)zb[0] * n + zb[1]] += 4.0 * t.coeff;
      }
      q0 = q1;
      continue;
    }
    int sq[32], ns = 0;  // support qubits (n <= 32)
    for (int q = 0; q < n; ++q)
      if ((x >> q) & 1ull) sq[ns++] = q;
    if (ns != 2 && ns != 4) return false;
    uint64_t zc = 0;  // the chains
    for (int i = 0; i < ns; i += 2)
      for (int q = sq[i] + 1; q < sq[i + 1]; ++q) zc |= 1ull << q;
    for (size_t k = q0; k < q1; ++k) {
      const uint64_t extra = (T[order[k]].z & ~x) ^ zc;
      if (extra && (ns == 4 || popc(extra) > 1)) return false;
    }
    // every flip direction: c occupies half the support, as many alpha and beta
    // qubits as it leaves empty
    for (int m = 0; m < (1 << ns); ++m) {
      uint64_t cd = 0;
      for (int i = 0; i < ns; ++i)
        if ((m >> i) & 1) cd |= 1ull << sq[i];
      if (2 * popc(cd & kEvenMask) != xe || 2 * popc(cd & ~kEvenMask) != xo) continue;
      // D(c) = (-1)^{xor of PP_c over S} * (-1)^{c_s1 ^ c_s3} * sum_t c_t i^y_t (-1)^{popc(z_t & S & ~c)} * ...
      const double pref = ((((cd >> sq[0]) ^ (ns == 4 ? (cd >> sq[2]) : 0ull)) & 1ull) ? -1.0 : 1.0);
      double w0 = 0.0;
      std::fill(wr.begin(), wr.end(), 0.0);
      for (size_t k = q0; k < q1; ++k) {
        const qf_term& t = T[order[k]];
        const int y = popc(t.x & t.z) & 3;  // 0 or 2
        double val = t.coeff * (y == 2 ? -1.0 : 1.0) * ((popc(t.z & x & ~cd) & 1) ? -1.0 : 1.0) * pref;
        const uint64_t extra = (t.z & ~x) ^ zc;
        if (!extra)
          w0 += val;
        else
          wr[__builtin_ctzll(extra)] += val;
      }
      int oc[2], em[2], noc = 0, nem = 0;  // occupied / empty support qubits of c (ns / 2 each)
      for (int i = 0; i < ns; ++i) {
        if ((cd >> sq[i]) & 1ull) oc[noc++] = sq[i];
        else em[nem++] = sq[i];
      }
      if (ns == 2) {
        const bool beta = oc[0] & 1;
        const int lo = oc[0] >> 1, lv = em[0] >> 1, nn = beta ? no : ne;
        double* row = (beta ? h->s1b.data() : h->s1a.data()) + (size_t)(lo * nn + lv) * (n + 1);
        double a = w0;
        for (int r = 0; r < n; ++r) {
          a += wr[r];
          row[1 + r] += -2.0 * wr[r];
        }
        row[0] += a;
      } else if (xe == 2) {
        int oa = -1, va = -1, ob = -1, vb = -1;
        for (int i = 0; i < noc; ++i) (oc[i] & 1 ? ob : oa) = oc[i] >> 1;
        for (int i = 0; i < nem; ++i) (em[i] & 1 ? vb : va) = em[i] >> 1;
        h->wab[(((size_t)oa * ne + va) * no + ob) * no + vb] += w0;
      } else {
        const int P = xe == 4 ? pe : po;
        (xe == 4 ? h->waa : h->wbb)[(size_t)pr(oc[0] >> 1, oc[1] >> 1) * P + pr(em[0] >> 1, em[1] >> 1)] += w0;
      }
    }
    q0 = q1;
  }
  return true;
}

// Builds and uploads a plan's direct tables on first use.
qf_status ensure_direct(qf_state* st, ExpPlan* p) {
  if (p->direct != 0) return QF_OK;
  DirectHost h;
  if (!build_direct(p->terms, st->n, &h)) {
    p->direct = -1;
    return QF_OK;
  }
  const int n = st->n;
  // fixed point: the largest sum of magnitudes any member can add stays below 2^61
  double bound = 0.0;
  for (double v : h.dg) bound += std::fabs(v);
  for (const std::vector<double>* t : {&h.s1a, &h.s1b})
    for (size_t r = 0; r < t->size(); r += n + 1) {
      double b = 0.0;
      for (int k = 0; k <= n; ++k) b += std::fabs((*t)[r + k]);
      bound = std::max(bound, b);
    }
  int e = 0;
  if (bound > 0.0) e = std::min(1000, 61 - (int)std::ceil(std::log2(bound)));
  auto to_fix = [&](const std::vector<double>& v) {
    std::vector<long long> o(v.size());
    for (size_t i = 0; i < v.size(); ++i) o[i] = std::llrint(std::ldexp(v[i], e));
    return o;
  };
  const std::vector<long long> f1a = to_fix(h.s1a), f1b = to_fix(h.s1b), fdg = to_fix(h.dg);
  auto f32 = [](const std::vector<double>& v) {
    std::vector<float> o(v.size());
    for (size_t i = 0; i < v.size(); ++i) o[i] = (float)v[i];
    return o;
  };
  const std::vector<float> fab = f32(h.wab), faa = f32(h.waa), fbb = f32(h.wbb);
  auto ds = [](const std::vector<double>& v) {  // (hi, lo) float pairs
    std::vector<float2> o(v.size());
    for (size_t i = 0; i < v.size(); ++i) {
      const float hi = (float)v[i];
      o[i] = make_float2(hi, (float)(v[i] - (double)hi));
    }
    return o;
  };
  const std::vector<float2> dab = ds(h.wab), daa = ds(h.waa), dbb = ds(h.wbb);
  // one buffer: doubles, floats, fixed point (each part 256-byte aligned)
  auto al = [](size_t b) { return (b + 255) / 256 * 256; };
  const size_t o_wab = 0, o_waa = o_wab + al(h.wab.size() * 8), o_wbb = o_waa + al(h.waa.size() * 8),
               o_fab = o_wbb + al(h.wbb.size() * 8), o_faa = o_fab + al(fab.size() * 4),
               o_fbb = o_faa + al(faa.size() * 4), o_s1a = o_fbb + al(fbb.size() * 4),
               o_s1b = o_s1a + al(f1a.size() * 8), o_dg = o_s1b + al(f1b.size() * 8),
               o_dab = o_dg + al(fdg.size() * 8), o_daa = o_dab + al(dab.size() * 8), o_dbb = o_daa + al(daa.size() * 8),
               total = o_dbb + al(dbb.size() * 8);
  std::vector<char> buf(total, 0);
  std::memcpy(buf.data() + o_wab, h.wab.data(), h.wab.size() * 8);
  std::memcpy(buf.data() + o_waa, h.waa.data(), h.waa.size() * 8);
  std::memcpy(buf.data() + o_wbb, h.wbb.data(), h.wbb.size() * 8);
  std::memcpy(buf.data() + o_fab, fab.data(), fab.size() * 4);
  std::memcpy(buf.data() + o_faa, faa.data(), faa.size() * 4);
  std::memcpy(buf.data() + o_fbb, fbb.data(), fbb.size() * 4);
  std::memcpy(buf.data() + o_s1a, f1a.data(), f1a.size() * 8);
  std::memcpy(buf.data() + o_s1b, f1b.data(), f1b.size() * 8);
  std::memcpy(buf.data() + o_dg, fdg.data(), fdg.size() * 8);
  std::memcpy(buf.data() + o_dab, dab.data(), dab.size() * 8);
  std::memcpy(buf.data() + o_daa, daa.data(), daa.size() * 8);
  std::memcpy(buf.data() + o_dbb, dbb.data(), dbb.size() * 8);
  if (cudaMalloc(&p->d_direct, total) != cudaSuccess) {
    cudaGetLastError();
    p->d_direct = nullptr;
    return fail(QF_ENOMEM, "cudaMalloc(direct H tables) failed");
  }
  QF_CUDA(h2d(p->d_direct, buf.data(), total, st->stream));
  QF_CUDA(cudaStreamSynchronize(st->stream));  // the staging buffer is freed on return
  char* b = static_cast<char*>(p->d_direct);
  qf::SecDirect& d = p->dtab;
  d.n = n;
  d.ne = (n + 1) / 2;
  d.no = n / 2;
  d.wab = reinterpret_cast<const double*>(b + o_wab);
  d.waa = reinterpret_cast<const double*>(b + o_waa);
  d.wbb = reinterpret_cast<const double*>(b + o_wbb);
  d.fab = reinterpret_cast<const float*>(b + o_fab);
  d.faa = reinterpret_cast<const float*>(b + o_faa);
  d.fbb = reinterpret_cast<const float*>(b + o_fbb);
  d.s1a = reinterpret_cast<const long long*>(b + o_s1a);
  d.s1b = reinterpret_cast<const long long*>(b + o_s1b);
  d.dg = reinterpret_cast<const long long*>(b + o_dg);
  d.dab = reinterpret_cast<const float2*>(b + o_dab);
  d.daa = reinterpret_cast<const float2*>(b + o_daa);
  d.dbb = reinterpret_cast<const float2*>(b + o_dbb);
  d.inv_fix = std::ldexp(1.0, -e);
  p->direct = 1;
  return QF_OK;
}

// Tables of the tiled H|psi> kernels, built the first time a plan needs them.
qf_status ensure_tiled(qf_state* st, ExpPlan* pp) {
  if (pp->tiled) return QF_OK;
  ExpPlan& p = *pp;
  const qf_term* terms = p.terms.data();
  std::map<uint64_t, std::vector<size_t>> byx;
  for (size_t i = 0; i < p.terms.size(); ++i) byx[terms[i].x].push_back(i);
  // tiled H|psi> tables: D_g(b) = sum_t c_t i^{y_t} s_t(b), eight terms per table
  std::vector<qf::HGroup> hg;
  std::vector<qf::WChunk> wc;
  std::vector<qf::WChunkF> wf;
  std::vector<qf::WChunkS> ws;
  for (auto& kv : byx) {
    qf::HGroup g{};
    g.x = kv.first;
    g.chunk0 = (int)wc.size();
    const std::vector<size_t>& idx = kv.second;
    g.nchunk = (int)((idx.size() + qf::kWideTerms - 1) / qf::kWideTerms);
    for (size_t k = 0; k < idx.size(); k += qf::kWideTerms) {
      qf::WChunk c{};
      qf::WChunkF cf{};
      qf::WChunkS cs{};
      const int cnt = (int)std::min<size_t>(qf::kWideTerms, idx.size() - k);
      for (int t = 0; t < qf::kWideTerms; ++t) c.z[t] = cf.z[t] = (t < cnt) ? terms[idx[k + t]].z : 0ull;
      // double-single tables (tiles of 2^12): split each term's pattern bit into a
      // tile part (z >> 12), a thread-nibble part and an element part.
      {
        const unsigned xhi = (unsigned)((kv.first >> 8) & 15u);
        for (int t = 0; t < qf::kWideTerms; ++t) cs.zh[t] = c.z[t] >> 12;
        for (int v = 0; v < 16; ++v) {
          unsigned bl = 0, bh = 0, bk = 0;
          for (int t = 0; t < qf::kWideTerms; ++t) {
            const uint64_t z = c.z[t];
            bl |= (unsigned)(popc(z & 15u & (uint64_t)v) & 1) << t;
            bh |= (unsigned)(popc(z & 0xF0u & ((uint64_t)v << 4)) & 1) << t;
            bk |= (unsigned)(popc((z >> 8) & 15u & (uint64_t)(v ^ xhi)) & 1) << t;
          }
          cs.nl[v] = (uint8_t)bl;
          cs.nh[v] = (uint8_t)bh;
          cs.kx[v] = (uint8_t)bk;
        }
      }
      for (int pat = 0; pat < (1 << qf::kWideTerms); ++pat) {
        double hx = 0, hy = 0;
        for (int t = 0; t < cnt; ++t) {
          const qf_term& T = terms[idx[k + t]];
          const int y = popc(T.x & T.z) & 3;
          const double c0 = ((pat >> t) & 1) ? -T.coeff : T.coeff;
          if ((y & 1) == 0)
            hx += c0 * ((y == 2) ? -1.0 : 1.0);
          else
            hy += c0 * ((y == 3) ? -1.0 : 1.0);
        }
        c.tab[pat] = make_double2(hx, hy);
        cf.tab[pat] = make_float2((float)hx, (float)hy);
        const float hh = (float)hx;
        cs.tab[pat] = make_float2(hh, (float)(hx - (double)hh));
      }
      for (int t = 0; t < cnt; ++t)
        if (popc(terms[idx[k + t]].x & terms[idx[k + t]].z) & 1) g.odd = 1;
      wc.push_back(c);
      wf.push_back(cf);
      ws.push_back(cs);
    }
    hg.push_back(g);
  }
  std::vector<qf::HClass> cls[qf::kClassTbN];
  for (int v = 0; v < qf::kClassTbN; ++v) {
    const int tb = qf::kClassTb0 + v;
    for (int g = 0; g < (int)hg.size(); ++g) {
      const uint64_t xh = hg[g].x >> tb;
      if (cls[v].empty() || cls[v].back().xh != xh) cls[v].push_back(qf::HClass{xh, g, g + 1});
      else cls[v].back().g1 = g + 1;
    }
    p.nclasses[v] = (int)cls[v].size();
  }
  if (cudaMalloc(&p.d_hgroups, std::max<size_t>(1, hg.size()) * sizeof(qf::HGroup)) != cudaSuccess ||
      cudaMalloc(&p.d_wchunks, std::max<size_t>(1, wc.size()) * sizeof(qf::WChunk)) != cudaSuccess ||
      cudaMalloc(&p.d_wchunks_f, std::max<size_t>(1, wf.size()) * sizeof(qf::WChunkF)) != cudaSuccess ||
      cudaMalloc(&p.d_wchunks_s, std::max<size_t>(1, ws.size()) * sizeof(qf::WChunkS)) != cudaSuccess ||
      cudaMalloc(&p.d_classes[0], std::max<size_t>(1, cls[0].size()) * sizeof(qf::HClass)) != cudaSuccess ||
      cudaMalloc(&p.d_classes[1], std::max<size_t>(1, cls[1].size()) * sizeof(qf::HClass)) != cudaSuccess ||
      cudaMalloc(&p.d_classes[2], std::max<size_t>(1, cls[2].size()) * sizeof(qf::HClass)) != cudaSuccess) {
    cudaGetLastError();
    return fail(QF_ENOMEM, "cudaMalloc(tiled plan) failed");
  }
  QF_CUDA(h2d(p.d_hgroups, hg.data(), hg.size() * sizeof(qf::HGroup), st->stream));
  QF_CUDA(h2d(p.d_wchunks, wc.data(), wc.size() * sizeof(qf::WChunk), st->stream));
  QF_CUDA(h2d(p.d_wchunks_f, wf.data(), wf.size() * sizeof(qf::WChunkF), st->stream));
  QF_CUDA(h2d(p.d_wchunks_s, ws.data(), ws.size() * sizeof(qf::WChunkS), st->stream));
  for (int v = 0; v < qf::kClassTbN; ++v)
    QF_CUDA(h2d(p.d_classes[v], cls[v].data(), cls[v].size() * sizeof(qf::HClass), st->stream));
  QF_CUDA(cudaStreamSynchronize(st->stream));
  p.tiled = true;
  return QF_OK;
}

// ---------------------------------------------------------------------------
// Sparse composite of a run of commuting rotations sharing one X mask.

struct RotIn {
  uint64_t x, z;
  double th;
  double coeff;  // generator weight for the gradient (coeff of the ansatz rotation)
};

bool commute(uint64_t x1, uint64_t z1, uint64_t x2, uint64_t z2) {
  return ((popc(x1 & z2) + popc(z1 & x2)) & 1) == 0;
}

// Build the composite on the support of x for every sign class.  On success
// fills a with M - I restricted to the active rows (M the forward composite,
// or its inverse when `inverse`) and, when `with_gen`, the generator
// Q = sum_k coeff_k P_k (whose rows then also count as active).
bool build_sparse(const RotIn* r, int m, int n, bool inverse, bool with_gen, qf::SparseArgs* a) {
  const uint64_t x = r[0].x;
  const int u = popc(x);
  if (u == 0 || u > qf::kSparseMaxSupp) return false;
  // scratch kept per thread (plan_blocks builds thousands of blocks in parallel)
  thread_local std::vector<int> supp, act;
  thread_local std::vector<uint64_t> zc;
  thread_local std::vector<cplx> dg, of, qg, pr;
  supp.clear();
  for (int i = 0; i < n; ++i)
    if ((x >> i) & 1) supp.push_back(i);
  auto compress = [&](uint64_t v) {
    uint64_t o = 0;
    for (int i = 0; i < u; ++i)
      if ((v >> supp[i]) & 1) o |= 1ull << i;
    return o;
  };
  zc.clear();
  for (int k = 0; k < m; ++k) {
    const uint64_t zo = r[k].z & ~x;
    if (zo && std::find(zc.begin(), zc.end(), zo) == zc.end()) zc.push_back(zo);
  }
  if (zc.size() > 2) return false;
  const int ncls = 1 << zc.size();
  const int D = 1 << u;
  const uint64_t xl = (uint64_t)D - 1;
  // Every rotation of the block pairs row with row ^ xl, so the composite M stays
  // block diagonal in those pairs and the generator Q only links a row to its
  // partner.  Per class, dg[row] = M[row][row], of[row] = M[row][row ^ xl] and
  // qg[row] = Q[row][row ^ xl] are the only entries that can differ from the
  // identity (every other entry of M - I and of Q stays exactly zero).
  dg.assign((size_t)ncls * D, cplx(1.0, 0.0));
  of.assign((size_t)ncls * D, cplx(0.0, 0.0));
  qg.assign((size_t)ncls * D, cplx(0.0, 0.0));
  pr.assign(D, cplx(0.0, 0.0));
  const cplx iu(0, 1);
  for (int c = 0; c < ncls; ++c) {
    cplx* M0 = &dg[(size_t)c * D];
    cplx* M1 = &of[(size_t)c * D];
    cplx* Q = &qg[(size_t)c * D];
    for (int k = 0; k < m; ++k) {
      const uint64_t zo = r[k].z & ~x;
      double sig = 1.0;
      if (zo) {
        const int j = (int)(std::find(zc.begin(), zc.end(), zo) - zc.begin());
        if ((c >> j) & 1) sig = -1.0;
      }
      const uint64_t zin = compress(r[k].z & x);
      const int y = popc(x & r[k].z) & 3;
      const cplx iy = (y == 0) ? cplx(1, 0) : (y == 1) ? cplx(0, 1) : (y == 2) ? cplx(-1, 0) : cplx(0, -1);
      // P|col> = iy (-1)^{popc(zin & col)} |col ^ xl>, times the class sign:
      // pr[row] is the coefficient of P in (row, row ^ xl)
      for (int row = 0; row < D; ++row)
        pr[row] = iy * sig * ((popc(zin & (uint64_t)(row ^ (int)xl)) & 1) ? -1.0 : 1.0);
      const double th = inverse ? -r[k].th : r[k].th;
      const double cs = std::cos(th), sn = std::sin(th);
      // only the 2x2 block of each pair changes
      for (int r0 = 0; r0 < D; ++r0) {
        const int r1 = r0 ^ (int)xl;
        if (r1 < r0) continue;
        const cplx m00 = M0[r0], m01 = M1[r0], m10 = M1[r1], m11 = M0[r1];
        const cplx f0 = iu * sn * pr[r0], f1 = iu * sn * pr[r1];
        M0[r0] = cs * m00 - f0 * m10;
        M1[r0] = cs * m01 - f0 * m11;
        M1[r1] = cs * m10 - f1 * m00;
        M0[r1] = cs * m11 - f1 * m01;
      }
      for (int row = 0; row < D; ++row) Q[row] += r[k].coeff * pr[row];
    }
  }
  // For the inverse the product above is R_m(-th_m)...R_1(-th_1); it equals the inverse of the
  // forward composite because the block's rotations commute.
  // A row is active when its row or column of M - I or of Q (every class) has an
  // entry: on the diagonal, or linking it to its partner.
  const double tol = 1e-14;
  auto off_identity = [&](const cplx& d) { return d != 0.0 && std::abs(d) > tol; };
  act.clear();
  for (int row = 0; row < D; ++row) {
    const int rp = row ^ (int)xl;
    bool a2 = false;
    for (int c = 0; c < ncls && !a2; ++c) {
      const cplx* M0 = &dg[(size_t)c * D];
      const cplx* M1 = &of[(size_t)c * D];
      const cplx* Q = &qg[(size_t)c * D];
      if (off_identity(M0[row] - 1.0) || off_identity(M1[row]) || off_identity(M1[rp]))
        a2 = true;
      else if (with_gen && (Q[row] != 0.0 || Q[rp] != 0.0))
        a2 = true;
    }
    if (a2) act.push_back(row);
  }
  const int nr = (int)act.size();
  if (nr == 0 || nr > qf::kSparseMaxRows || 2 * nr > D) return false;
  std::memset(a, 0, sizeof(*a));
  a->u = u;
  a->nr = nr;
  a->ncls = ncls;
  a->nzc = (int)zc.size();
  for (int i = 0; i < u; ++i) a->supp[i] = supp[i];
  for (size_t j = 0; j < zc.size(); ++j) a->zc[j] = zc[j];
  for (int i = 0; i < nr; ++i) {
    uint64_t off = 0;
    for (int b = 0; b < u; ++b)
      if ((act[i] >> b) & 1) off |= 1ull << supp[b];
    a->pat[i] = off;
  }
  for (int c = 0; c < ncls; ++c)
    for (int i = 0; i < nr; ++i)
      for (int j = 0; j < nr; ++j) {
        const int ri = act[i], rj = act[j];
        const bool pair = rj == (ri ^ (int)xl);
        const cplx me = (rj == ri) ? dg[(size_t)c * D + ri] : pair ? of[(size_t)c * D + ri] : cplx(0.0, 0.0);
        const cplx mv = me - ((i == j) ? 1.0 : 0.0);
        const cplx qv = pair ? qg[(size_t)c * D + ri] : cplx(0.0, 0.0);
        a->M[c][i][j] = make_double2(mv.real(), mv.imag());
        a->Q[c][i][j] = make_double2(qv.real(), qv.imag());
      }
  return true;
}

// Recompute M - I of a sparse block for new angles, on its active rows only.
// This is exact: every rotation of the block pairs support pattern r with
// r ^ x, and the active rows are a union of such pairs, so each rotation maps
// the active rows onto themselves and the composite restricted to them is the
// product of the restricted rotations.
// The composites of a block's rotations r[0..m) (inverse: of the inverse rotations;
// a block's rotations commute) for its rows and sign classes in a: store(c, i, j, d)
// receives entry (i, j) of class c's composite minus the identity.  Reads only
// a's structure (rows, support, classes).
template <typename Store>
void compose_sparse(const RotIn* r, int m, bool inverse, const qf::SparseArgs& sa, Store&& store) {
  const qf::SparseArgs* a = &sa;
  const int u = a->u, nr = a->nr;
  const uint64_t x = r[0].x;
  const int xl = (1 << u) - 1;
  int loc[qf::kSparseMaxRows];
  for (int i = 0; i < nr; ++i) {
    int v = 0;
    for (int b = 0; b < u; ++b)
      if ((a->pat[i] >> a->supp[b]) & 1) v |= 1 << b;
    loc[i] = v;
  }
  int partner[qf::kSparseMaxRows];
  for (int i = 0; i < nr; ++i) {
    partner[i] = -1;
    for (int j = 0; j < nr; ++j)
      if (loc[j] == (loc[i] ^ xl)) partner[i] = j;
  }
  auto compress = [&](uint64_t v) {
    uint64_t o = 0;
    for (int b = 0; b < u; ++b)
      if ((v >> a->supp[b]) & 1) o |= 1ull << b;
    return o;
  };
  const cplx iu(0, 1);
  const int ncls = 1 << a->nzc;
  // phase pe of rotation k on row i in class c: P_k maps row i to its partner
  // with this factor (Y phase, outside-Z class sign, inside-Z parity)
  auto phase = [&](int k, int c, int i) {
    const uint64_t zo = r[k].z & ~x;
    double sig = 1.0;
    for (int j = 0; j < a->nzc; ++j)
      if (zo == a->zc[j] && ((c >> j) & 1)) sig = -1.0;
    const uint64_t zin = compress(r[k].z & x);
    const int y = popc(x & r[k].z) & 3;
    const cplx iy = (y == 0) ? cplx(1, 0) : (y == 1) ? cplx(0, 1) : (y == 2) ? cplx(-1, 0) : cplx(0, -1);
    const int col = loc[i] ^ xl;
    return iy * sig * ((popc(zin & (uint64_t)col) & 1) ? -1.0 : 1.0);
  };
  // Two rows: each rotation is cos(th) I - i sin(th) P_k on the pair.  When every
  // P_k is +-P_0 there (same phases up to one common sign per rotation), they
  // compose to cos(phi) I - i sin(phi) P_0 with phi the signed sum of the angles:
  // one sine and cosine per class instead of one per rotation and a product each.
  if (nr == 2 && partner[0] == 1 && partner[1] == 0) {
    bool closed = true;
    double phi[4] = {0.0, 0.0, 0.0, 0.0};
    cplx p0[4], p1[4];
    for (int c = 0; c < ncls && closed; ++c) {
      p0[c] = phase(0, c, 0);
      p1[c] = phase(0, c, 1);
      for (int k = 0; k < m && closed; ++k) {
        const cplx q0 = phase(k, c, 0), q1 = phase(k, c, 1);
        const double th = inverse ? -r[k].th : r[k].th;
        if (q0 == p0[c] && q1 == p1[c])
          phi[c] += th;
        else if (q0 == -p0[c] && q1 == -p1[c])
          phi[c] -= th;
        else
          closed = false;
      }
    }
    if (closed) {
      for (int c = 0; c < ncls; ++c) {
        const double cs = std::cos(phi[c]), sn = std::sin(phi[c]);
        store(c, 0, 0, cplx(cs - 1.0, 0.0));
        store(c, 0, 1, -iu * sn * p0[c]);
        store(c, 1, 0, -iu * sn * p1[c]);
        store(c, 1, 1, cplx(cs - 1.0, 0.0));
      }
      return;
    }
  }
  // one sine and cosine per rotation (a block's runs are short; longer ones spill to the heap)
  double cs_buf[32], sn_buf[32];
  std::vector<double> cs_heap, sn_heap;
  double* csv = cs_buf;
  double* snv = sn_buf;
  if (m > 32) {
    cs_heap.resize(m);
    sn_heap.resize(m);
    csv = cs_heap.data();
    snv = sn_heap.data();
  }
  for (int k = 0; k < m; ++k) {
    const double th = inverse ? -r[k].th : r[k].th;
    csv[k] = std::cos(th);
    snv[k] = std::sin(th);
  }
  for (int c = 0; c < ncls; ++c) {
    cplx M[qf::kSparseMaxRows][qf::kSparseMaxRows];
    for (int i = 0; i < nr; ++i)
      for (int j = 0; j < nr; ++j) M[i][j] = (i == j) ? 1.0 : 0.0;
    for (int k = 0; k < m; ++k) {
      const uint64_t zo = r[k].z & ~x;
      double sig = 1.0;
      for (int j = 0; j < a->nzc; ++j)
        if (zo == a->zc[j] && ((c >> j) & 1)) sig = -1.0;
      const uint64_t zin = compress(r[k].z & x);
      const int y = popc(x & r[k].z) & 3;
      const cplx iy = (y == 0) ? cplx(1, 0) : (y == 1) ? cplx(0, 1) : (y == 2) ? cplx(-1, 0) : cplx(0, -1);
      const double cs = csv[k], sn = snv[k];
      cplx N2[qf::kSparseMaxRows][qf::kSparseMaxRows];
      for (int i = 0; i < nr; ++i) {
        const int col = loc[i] ^ xl;
        const cplx pe = iy * sig * ((popc(zin & (uint64_t)col) & 1) ? -1.0 : 1.0);
        for (int j = 0; j < nr; ++j) N2[i][j] = cs * M[i][j] - iu * sn * pe * M[partner[i]][j];
      }
      for (int i = 0; i < nr; ++i)
        for (int j = 0; j < nr; ++j) M[i][j] = N2[i][j];
    }
    for (int i = 0; i < nr; ++i)
      for (int j = 0; j < nr; ++j) store(c, i, j, M[i][j] - ((i == j) ? 1.0 : 0.0));
  }
}

void refill_sparse(const RotIn* r, int m, bool inverse, qf::SparseArgs* a) {
  compose_sparse(r, m, inverse, *a,
                 [a](int c, int i, int j, cplx d) { a->M[c][i][j] = make_double2(d.real(), d.imag()); });
}

// The inverse block's composites as the adjoints of the forward block's (the
// composites are unitary), when both blocks list the same rows and sign classes:
// inv.M[c] = (f.M[c] + I)^dagger - I.  Returns false (nothing written) otherwise.
bool adjoint_composite(const qf::SparseArgs& f, qf::SparseArgs* inv) {
  if (f.nr != inv->nr || f.nzc != inv->nzc) return false;
  for (int i = 0; i < f.nr; ++i)
    if (f.pat[i] != inv->pat[i]) return false;
  for (int j = 0; j < f.nzc; ++j)
    if (f.zc[j] != inv->zc[j]) return false;
  const int ncls = 1 << f.nzc;
  for (int c = 0; c < ncls; ++c)
    for (int i = 0; i < f.nr; ++i)
      for (int j = 0; j < f.nr; ++j) {
        const double2 a = f.M[c][j][i];  // the identity's diagonal is real: M - I keeps its shape
        inv->M[c][i][j] = make_double2(a.x, -a.y);
      }
  return true;
}

// Largest m of the binomial table.  Every caller takes m <= n / 2 (orbitals of
// one spin) with n <= QF_MAX_QUBITS, and C(33, k) < 2^31, so the table's values
// are exact in 32 bits and its running products (< 2^36) cannot overflow.
constexpr int kBinomMax = 33;
static_assert(QF_MAX_QUBITS / 2 <= kBinomMax, "binomial table too small for QF_MAX_QUBITS");

uint32_t binom_loop(int m, int k) {
  if (k < 0 || k > m) return 0;
  uint64_t c = 1;
  for (int j = 1; j <= k; ++j) c = c * (uint64_t)(m - k + j) / (uint64_t)j;
  return (uint32_t)c;
}

// C(m, k) for 0 <= m <= kBinomMax from a table filled once by the same loop;
// 0 for k outside 0..m.  An m outside the table is a planning error: it gives
// 0 (never a truncated value) and is caught by qf_state_create's qubit limit
// before any caller can reach it.
uint32_t binom(int m, int k) {
  struct Table {
    uint32_t v[kBinomMax + 1][kBinomMax + 1];
    Table() {
      for (int i = 0; i <= kBinomMax; ++i)
        for (int j = 0; j <= kBinomMax; ++j) v[i][j] = binom_loop(i, j);
    }
  };
  static const Table t;  // thread-safe one-time initialisation
  if (m < 0 || m > kBinomMax || k < 0 || k > m) return 0;
  return t.v[m][k];
}

// The real composite-minus-identity m and, for an inverse block, the real Qi of
// its generator Q = i Qi, per sign class, of a two-row block; false when the
// block is not of that form.  The reverse sweep takes Qi = [[0, q01], [-q01, 0]]
// (the generator only links the two active patterns).
bool sector_mq(const qf::SparseArgs& a, bool need_q, double (*m)[2][2], double (*q)[2][2]) {
  if (a.nr != 2) return false;
  const int ncls = 1 << a.nzc;
  for (int c = 0; c < ncls; ++c)
    for (int i = 0; i < 2; ++i)
      for (int j = 0; j < 2; ++j) {
        if (a.M[c][i][j].y != 0.0) return false;
        if (need_q && a.Q[c][i][j].x != 0.0) return false;
      }
  if (need_q)
    for (int c = 0; c < ncls; ++c)
      if (a.Q[c][0][0].y != 0.0 || a.Q[c][1][1].y != 0.0 || a.Q[c][1][0].y != -a.Q[c][0][1].y) return false;
  for (int c = 0; c < qf::kSparseMaxCls; ++c)
    for (int i = 0; i < 2; ++i)
      for (int j = 0; j < 2; ++j) {
        const int cc = c < ncls ? c : 0;
        m[c][i][j] = a.M[cc][i][j].x;
        q[c][i][j] = need_q ? a.Q[cc][i][j].y : 0.0;
      }
  return true;
}

// A two-row sparse block as a sector block for a state with (na, nb) occupied
// even/odd qubits.  Requires a real composite, two active patterns with equal
// even and odd occupation (so the block maps the sector onto itself) and, for
// the reverse sweep, a purely imaginary generator.  A block that no member can
// carry is accepted with zero items (it acts as the identity on the sector).
bool to_secblk(const qf::SparseArgs& a, int n, int na, int nb, bool need_q, qf::SecBlk* o) {
  if (a.nr != 2 || n > 2 * qf::kSecMaxPos) return false;
  const uint64_t p0 = a.pat[0], p1 = a.pat[1];
  const int e0 = popc(p0 & kEvenMask), o0 = popc(p0 & ~kEvenMask);
  if (e0 != popc(p1 & kEvenMask) || o0 != popc(p1 & ~kEvenMask)) return false;
  std::memset(o, 0, sizeof(*o));
  if (!sector_mq(a, need_q, o->m, o->q)) return false;
  uint64_t U = 0;
  for (int i = 0; i < a.u; ++i) U |= 1ull << a.supp[i];
  for (int q = 0; q < n; ++q) {
    if ((U >> q) & 1) continue;
    if ((q & 1) == 0)
      o->epos[o->ne++] = (uint8_t)q;
    else
      o->opos[o->no++] = (uint8_t)q;
  }
  // a block whose patterns no member of the sector can carry (too few or too
  // many electrons left for the outside positions) touches nothing: zero items
  o->ke = na - e0;
  o->ko = nb - o0;
  o->cnt_e = binom(o->ne, o->ke);
  o->cnt_o = binom(o->no, o->ko);
  o->pat[0] = p0;
  o->pat[1] = p1;
  o->zc[0] = a.zc[0];
  o->zc[1] = a.zc[1];
  o->nzc = a.nzc;
  return true;
}

qf::SecSpace sector_space(int n, int na, int nb) {
  qf::SecSpace sp{};
  for (int q = 0; q < n; ++q) {
    if ((q & 1) == 0)
      sp.epos[sp.ne++] = (uint8_t)q;
    else
      sp.opos[sp.no++] = (uint8_t)q;
  }
  sp.ke = na;
  sp.ko = nb;
  sp.cnt_e = binom(sp.ne, na);
  sp.cnt_o = binom(sp.no, nb);
  return sp;
}

// Colex rank of a k-subset mask among all k-subsets: sum over its set bits,
// taken in increasing position p_1 < p_2 < ..., of C(p_i, i).
uint32_t colex_rank(uint32_t mask) {
  uint32_t r = 0;
  int i = 0;
  for (int p = 0; p < 32; ++p)
    if ((mask >> p) & 1u) r += binom(p, ++i);
  return r;
}

// Compact index of basis state det in its sector (SecCompact ordering).
uint64_t compact_of(uint64_t det, const qf::SecSpace& sp) {
  return (uint64_t)colex_rank(local_bits(det, 0)) * sp.cnt_o + colex_rank(local_bits(det, 1));
}

// Rank tables of sector (na, nb) and a compact buffer of 2 * members amplitudes.
qf_status ensure_compact(qf_state* st, const qf::SecSpace& sp, int na, int nb, qf::SecCompact* cm) {
  const size_t ea = (size_t)1 << sp.ne, eb = (size_t)1 << sp.no;
  if (st->rank_n != st->n || st->rank_a != na || st->rank_b != nb) {
    // every mask's colex rank among the masks of its own popcount (the part-local
    // sweeps rank strings of other electron counts with the same table)
    std::vector<uint16_t> t(ea + eb);
    for (size_t m = 0; m < ea; ++m) t[m] = (uint16_t)colex_rank((uint32_t)m);
    for (size_t m = 0; m < eb; ++m) t[ea + m] = (uint16_t)colex_rank((uint32_t)m);
    cudaFree(st->d_rank);
    st->d_rank = nullptr;
    st->rank_n = -1;
    if (cudaMalloc(&st->d_rank, t.size() * sizeof(uint16_t)) != cudaSuccess) {
      cudaGetLastError();
      st->d_rank = nullptr;
      return fail(QF_ENOMEM, "cudaMalloc(sector rank tables) failed");
    }
    QF_CUDA(h2d(st->d_rank, t.data(), t.size() * sizeof(uint16_t), st->stream));
    st->rank_n = st->n;
    st->rank_a = na;
    st->rank_b = nb;
  }
  const size_t need = 2 * (size_t)sp.cnt_e * sp.cnt_o * st->elem();
  if (need > st->cstate_cap) {
    cudaFree(st->d_cstate);
    st->d_cstate = nullptr;
    st->cstate_cap = 0;
    if (cudaMalloc(&st->d_cstate, need) != cudaSuccess) {
      cudaGetLastError();
      st->d_cstate = nullptr;
      return fail(QF_ENOMEM, "cudaMalloc(compact sector state) failed");
    }
    st->cstate_cap = need;
  }
  cm->ra = st->d_rank;
  cm->rb = st->d_rank + ea;
  cm->cnt_o = sp.cnt_o;
  return QF_OK;
}

// Part-local runs (qf::RunInfo) for sector blocks sec[0..nblk) (forward) and
// sec[nblk..2 nblk) (their inverses) of an n-qubit state in sector (na, nb):
// consecutive blocks are grouped while the largest part of the union of their
// supports stays within cap members (and a run holds at most kRunMaxBlocks).

// Largest part of a run touching ua of the ne alpha and ub of the no beta orbitals.
uint64_t run_maxpart(int ua, int ub, int ne, int no, int na, int nb) {
  uint64_t ba = 0, bb = 0;
  for (int ka = std::max(0, na - (ne - ua)); ka <= std::min(ua, na); ++ka) ba = std::max<uint64_t>(ba, binom(ua, ka));
  for (int kb = std::max(0, nb - (no - ub)); kb <= std::min(ub, nb); ++kb) bb = std::max<uint64_t>(bb, binom(ub, kb));
  return ba * bb;
}

bool build_runs(const qf::SecBlk* sec, size_t nblk, int n, int na, int nb, uint64_t cap, SectorRuns* out) {
  const int ne = (n + 1) / 2, no = n / 2;
  const uint64_t all = (n >= 64) ? ~0ull : ((1ull << n) - 1);
  std::vector<uint64_t> supp(nblk);
  for (size_t b = 0; b < nblk; ++b) {
    uint64_t outside = 0;
    for (int i = 0; i < sec[b].ne; ++i) outside |= 1ull << sec[b].epos[i];
    for (int i = 0; i < sec[b].no; ++i) outside |= 1ull << sec[b].opos[i];
    supp[b] = all & ~outside;
  }
  out->runs.clear();
  out->parts.clear();
  out->blks.assign(2 * nblk, qf::RunBlk{});
  out->pmax = 0;
  out->logitems = 0;
  out->run_items.clear();
  out->strs.clear();
  out->log_ok = true;
  for (size_t b = 0; b < nblk; ++b)
    if (sec[b].pat[0] != sec[nblk + b].pat[0] || sec[b].pat[1] != sec[nblk + b].pat[1]) out->log_ok = false;
  size_t b0 = 0;
  while (b0 < nblk) {
    uint64_t U = supp[b0];
    size_t b1 = b0 + 1;
    while (b1 < nblk && b1 - b0 < (size_t)qf::kRunMaxBlocks) {
      const uint64_t U2 = U | supp[b1];
      const int ua2 = popc(U2 & kEvenMask), ub2 = popc(U2 & ~kEvenMask);
      if (ua2 > qf::kRunMaxOrb || ub2 > qf::kRunMaxOrb || run_maxpart(ua2, ub2, ne, no, na, nb) > cap) break;
      U = U2;
      ++b1;
    }
    const int ua = popc(U & kEvenMask), ub = popc(U & ~kEvenMask);
    if (ua > qf::kRunMaxOrb || ub > qf::kRunMaxOrb || run_maxpart(ua, ub, ne, no, na, nb) > cap)
      return false;  // one block's own part too large
    qf::RunInfo R{};
    R.b0 = (int)b0;
    R.b1 = (int)b1;
    R.ua = ua;
    R.ub = ub;
    int loca[32] = {0}, locb[32] = {0};  // spin-local orbital -> run-local index
    uint32_t Ga = 0, Gb = 0;             // spin-local masks of G
    {
      int ia = 0, ib = 0;
      for (int q = 0; q < n; ++q) {
        const int orb = q >> 1;
        if ((U >> q) & 1ull) {
          if ((q & 1) == 0) {
            R.apos[ia] = (uint8_t)orb;
            loca[orb] = ia++;
          } else {
            R.bpos[ib] = (uint8_t)orb;
            locb[orb] = ib++;
          }
        } else if ((q & 1) == 0) {
          Ga |= 1u << orb;
        } else {
          Gb |= 1u << orb;
        }
      }
    }
    // parts: every occupation of G that leaves a feasible count on U, largest first
    std::vector<uint32_t> gas, gbs;
    for (uint32_t m = Ga;; m = (m - 1) & Ga) {
      const int ka = na - popc(m);
      if (ka >= 0 && ka <= ua) gas.push_back(m);
      if (m == 0) break;
    }
    for (uint32_t m = Gb;; m = (m - 1) & Gb) {
      const int kb = nb - popc(m);
      if (kb >= 0 && kb <= ub) gbs.push_back(m);
      if (m == 0) break;
    }
    std::vector<qf::RunPart> ps;
    ps.reserve(gas.size() * gbs.size());
    for (uint32_t ga : gas)
      for (uint32_t gb : gbs) {
        qf::RunPart P{};
        P.ga = ga;
        P.gb = gb;
        P.ka = na - popc(ga);
        P.kb = nb - popc(gb);
        P.cnta = binom(ua, P.ka);
        P.cntb = binom(ub, P.kb);
        ps.push_back(P);
      }
    std::stable_sort(ps.begin(), ps.end(), [](const qf::RunPart& a, const qf::RunPart& b) {
      return (uint64_t)a.cnta * a.cntb > (uint64_t)b.cnta * b.cntb;
    });
    R.part0 = (int)out->parts.size();
    R.nparts = (int)ps.size();
    R.maxsize = ps.empty() ? 0u : ps[0].cnta * ps[0].cntb;
    out->parts.insert(out->parts.end(), ps.begin(), ps.end());
    out->pmax = std::max(out->pmax, R.nparts);
    // the run's blocks in run-local coordinates (forward and inverse share the geometry)
    auto runlocal = [&](uint64_t mask, int par) {
      uint32_t o = 0;
      for (int q = par; q < n; q += 2)
        if (((mask >> q) & 1ull) && ((U >> q) & 1ull)) o |= 1u << (par ? locb[q >> 1] : loca[q >> 1]);
      return o;
    };
    for (size_t b = b0; b < b1; ++b)
      for (int dir = 0; dir < 2; ++dir) {
        const qf::SecBlk& S = sec[dir * nblk + b];
        qf::RunBlk& B = out->blks[dir * nblk + b];
        const uint64_t sp = supp[b];
        for (int q = 0; q < n; ++q) {
          if (!((U >> q) & 1ull) || ((sp >> q) & 1ull)) continue;
          if ((q & 1) == 0)
            B.epos[B.ne++] = (uint8_t)loca[q >> 1];
          else
            B.opos[B.no++] = (uint8_t)locb[q >> 1];
        }
        B.e0 = popc(S.pat[0] & kEvenMask);
        B.o0 = popc(S.pat[0] & ~kEvenMask);
        B.nzc = S.nzc;
        B.np = R.nparts;
        for (int i = 0; i < 2; ++i)
          for (int par = 0; par < 2; ++par) {
            B.pu[i][par] = runlocal(S.pat[i], par);
            B.zu[i][par] = runlocal(S.zc[i] & ~sp, par);
            B.zg[i][par] = local_bits(S.zc[i] & ~U, par);
          }
        std::memcpy(B.m, S.m, sizeof(B.m));
        std::memcpy(B.q, S.q, sizeof(B.q));
        qf::runblk_f32(B);
      }
    // forward-log layout: each part's items, block after block, parts in order.
    // Blocks of equal shape (outside counts, pattern electrons) share their count.
    std::map<std::array<int, 4>, uint64_t> shapes;
    for (size_t b = b0; b < b1; ++b) {
      const qf::RunBlk& B = out->blks[b];
      ++shapes[{B.ne, B.no, B.e0, B.o0}];
    }
    std::map<std::pair<int, int>, uint64_t> classes;  // (ka, kb) -> map base
    const uint64_t items0 = out->logitems;
    for (int k = 0; k < R.nparts; ++k) {
      qf::RunPart& P = out->parts[R.part0 + k];
      uint64_t tot = 0;
      for (const auto& sh : shapes) {
        const auto& f = sh.first;
        tot += sh.second * (uint64_t)binom(f[0], P.ka - f[2]) * binom(f[1], P.kb - f[3]);
      }
      P.logbase = out->logitems;
      out->logitems += tot;
      // parts with the same electron counts on U share one item map
      const auto seen = classes.find({P.ka, P.kb});
      P.maprep = seen == classes.end();
      P.mapbase = P.maprep ? out->mapwords : seen->second;
      if (P.maprep) {
        classes.emplace(std::make_pair(P.ka, P.kb), P.mapbase);
        out->mapwords += tot;
      }
    }
    out->runs.push_back(R);
    out->run_items.push_back(out->logitems - items0);
    b0 = b1;
  }
  // maps serve the reverse sweep too when each inverse block has its forward
  // block's item geometry (outside orbitals, patterns, class masks)
  out->map_ok = out->log_ok;
  for (const qf::RunInfo& R : out->runs)
    if (R.maxsize > qf::kMapMaxPart) out->map_ok = false;
  for (size_t b = 0; b < nblk && out->map_ok; ++b) {
    const qf::RunBlk& F = out->blks[b];
    const qf::RunBlk& I = out->blks[nblk + b];
    out->map_ok = F.ne == I.ne && F.no == I.no && F.e0 == I.e0 && F.o0 == I.o0 && F.nzc == I.nzc &&
                  std::memcmp(F.epos, I.epos, sizeof(F.epos)) == 0 && std::memcmp(F.opos, I.opos, sizeof(F.opos)) == 0 &&
                  std::memcmp(F.pu, I.pu, sizeof(F.pu)) == 0 && std::memcmp(F.zu, I.zu, sizeof(F.zu)) == 0 &&
                  std::memcmp(F.zg, I.zg, sizeof(F.zg)) == 0;
  }
  // outside strings of every block: all subsets of its outside positions, by size,
  // each size in colex order (= increasing mask), as run-local masks; shared by a
  // block and its inverse.  Left out when the table would pass kStringsMax entries.
  uint64_t total = 0;
  for (size_t b = 0; b < nblk; ++b) total += (1ull << out->blks[b].ne) + (1ull << out->blks[b].no);
  const bool tab = total <= kStringsMax;
  if (!tab) {
    for (size_t b = 0; b < 2 * nblk; ++b) out->blks[b].lsa = out->blks[b].lsb = qf::kNoStrings;
    return true;
  }
  // each block's two tables start where the previous blocks' end; filled in parallel
  std::vector<uint32_t> base(2 * nblk + 1, 0);
  for (size_t b = 0; b < nblk; ++b) {
    base[2 * b + 1] = base[2 * b] + (1u << out->blks[b].ne);
    base[2 * b + 2] = base[2 * b + 1] + (1u << out->blks[b].no);
  }
  out->strs.assign(base[2 * nblk], 0);
  qf::HostPool::get().parallel_for(nblk, 16, [&](size_t b) {
    qf::RunBlk& F = out->blks[b];
    qf::RunBlk& I = out->blks[nblk + b];
    for (int spin = 0; spin < 2; ++spin) {
      const int m = spin ? F.no : F.ne;
      const uint8_t* pos = spin ? F.opos : F.epos;
      const uint32_t b0 = base[2 * b + spin];
      uint32_t next[qf::kSecMaxPos + 1];  // next slot of each size
      uint32_t acc = b0;
      for (int k = 0; k <= m; ++k) {
        next[k] = acc;
        acc += binom(m, k);
      }
      for (uint32_t mask = 0; mask < (1u << m); ++mask) {
        uint32_t dep = 0;
        for (int j = 0; j < m; ++j)
          if ((mask >> j) & 1u) dep |= 1u << pos[j];
        out->strs[next[popc(mask)]++] = (uint16_t)dep;
      }
      (spin ? F.lsb : F.lsa) = b0;
      (spin ? I.lsb : I.lsa) = b0;
    }
  });
  return true;
}

// A device buffer of at least `bytes`, kept with the handle.
qf_status ensure_buf(void** p, size_t* cap, size_t bytes, const char* what) {
  if (bytes <= *cap) return QF_OK;
  cudaFree(*p);
  *p = nullptr;
  *cap = 0;
  if (cudaMalloc(p, bytes) != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return fail(QF_ENOMEM, std::string("cudaMalloc(") + what + ") failed");
  }
  *cap = bytes;
  return QF_OK;
}

// Residual read-out: out[2k], out[2k + 1] = the amplitude of lam at idx[k].
cudaError_t gather_residuals(qf_state* st, const void* lam, bool packed, bool ds, const std::vector<int64_t>& idx,
                             double* out) {
  if (ensure_buf(&st->d_idx, &st->idx_cap, idx.size() * sizeof(int64_t), "residual indices") != QF_OK)
    return cudaErrorMemoryAllocation;
  cudaError_t e = h2d(st->d_idx, idx.data(), idx.size() * sizeof(int64_t), st->stream);
  if (e != cudaSuccess) return e;
  return qf::launch_gather(lam, st->dt, static_cast<const int64_t*>(st->d_idx), (int)idx.size(), packed, ds, out,
                           st->stream);
}

qf_status ensure_sector_buffers(qf_state* st, size_t nblk, size_t partials) {
  if (nblk > st->secblk_cap) {
    cudaFree(st->d_secblk);
    st->d_secblk = nullptr;
    st->secblk_cap = 0;
    if (cudaMalloc(&st->d_secblk, nblk * sizeof(qf::SecBlk)) != cudaSuccess) {
      cudaGetLastError();
      return fail(QF_ENOMEM, "cudaMalloc(sector blocks) failed");
    }
    st->secblk_cap = nblk;
  }
  if (partials > st->sec_partial_cap) {
    cudaFree(st->d_sec_partial);
    st->d_sec_partial = nullptr;
    st->sec_partial_cap = 0;
    if (cudaMalloc(&st->d_sec_partial, partials * sizeof(double)) != cudaSuccess) {
      cudaGetLastError();
      return fail(QF_ENOMEM, "cudaMalloc(sector partials) failed");
    }
    st->sec_partial_cap = partials;
  }
  if (!st->d_bar) {
    if (cudaMalloc(&st->d_bar, 4 * sizeof(unsigned)) != cudaSuccess) {
      cudaGetLastError();
      return fail(QF_ENOMEM, "cudaMalloc(barrier) failed");
    }
  }
  return QF_OK;
}

// Reads the sweep's error flag (grid barrier timeout) after the stream synchronised.
qf_status check_barrier(qf_state* st) {
  unsigned flags[3] = {0, 0, 0};
  QF_CUDA(cudaMemcpyAsync(flags, st->d_bar, sizeof(flags), cudaMemcpyDeviceToHost, st->stream));
  QF_CUDA(cudaStreamSynchronize(st->stream));
  if (flags[2]) return fail(QF_ETIMEOUT, "sector sweep: grid barrier wait exceeded its limit");
  return QF_OK;
}

// Length of the run starting at i that can form one sparse block.
int sparse_run(const RotIn* r, size_t i, size_t nrot, const int32_t* params) {
  const uint64_t x = r[i].x;
  if (x == 0) return 1;
  size_t j = i + 1;
  while (j < nrot && r[j].x == x && (!params || params[j] == params[i])) {
    bool ok = true;
    for (size_t k = i; k < j && ok; ++k) ok = commute(r[k].x, r[k].z, r[j].x, r[j].z);
    if (!ok) break;
    ++j;
  }
  return (int)(j - i);
}

// Fill a TileArgs for rotations [i, j) whose X union fits the tile.
void build_tile(qf_state* st, const RotIn* r, size_t i, size_t j, uint64_t uni, qf::TileArgs* a) {
  const int n = st->n;
  const int s_target = std::min(n, st->dt == QF_C128 ? 11 : 12);
  uint64_t S = uni;
  for (int b = 0; b < n && popc(S) < s_target; ++b) S |= 1ull << b;
  std::memset(a, 0, sizeof(*a));
  a->s = popc(S);
  int l = 0;
  while (l < n && ((S >> l) & 1)) ++l;
  a->l = l;
  a->nhi = a->s - l;
  int k = 0, kh = 0;
  for (int b = 0; b < n; ++b)
    if ((S >> b) & 1) {
      a->sbits[k++] = b;
      if (b >= l) a->pos[kh++] = b;
    }
  auto compress = [&](uint64_t v) {
    uint32_t o = 0;
    for (int q = 0; q < a->s; ++q)
      if ((v >> a->sbits[q]) & 1) o |= 1u << q;
    return o;
  };
  a->m = (int)(j - i);
  for (size_t t = i; t < j; ++t) {
    qf::TileRot& R = a->r[t - i];
    R.xl = compress(r[t].x);
    R.zl = compress(r[t].z & S);
    R.zout = r[t].z & ~S;
    R.hl = r[t].x ? 31 - __builtin_clz(R.xl) : -1;
    R.y = popc(r[t].x & r[t].z);
    rot_coeffs(st->dt, &st->scale, r[t].th, &R.form, &R.A, &R.B);
  }
}

uint64_t typical_items(const qf::SecBlk* b, size_t n) {
  std::vector<uint64_t> v(n);
  for (size_t i = 0; i < n; ++i) v[i] = (uint64_t)b[i].cnt_e * b[i].cnt_o;
  std::nth_element(v.begin(), v.begin() + n / 2, v.end());
  return n ? v[n / 2] : 1;
}

qf_status flush_sector(qf_state* st, std::vector<qf::SecBlk>& pend) {
  if (pend.empty()) return QF_OK;
  const int grid = qf::sector_sweep_grid(typical_items(pend.data(), pend.size()));
  qf_status bs = ensure_sector_buffers(st, pend.size(), 1);
  if (bs != QF_OK) return bs;
  QF_CUDA(h2d(st->d_secblk, pend.data(), pend.size() * sizeof(qf::SecBlk), st->stream));
  QF_CUDA(qf::launch_sector_sweep(st->psi, st->dt, st->real, st->d_secblk, (int)pend.size(), st->d_bar, grid,
                                  st->stream));
  QF_CUDA(cudaStreamSynchronize(st->stream));  // the descriptor buffer is reused by the next flush
  pend.clear();
  return check_barrier(st);
}

qf_status apply_rotations(qf_state* st, const RotIn* r, size_t nrot) {
  const int n = st->n;
  const int umax = std::min(n, 8);
  std::vector<qf::SecBlk> pend;  // sector blocks waiting for one sweep launch
  size_t i = 0;
  while (i < nrot) {
    const int run = sparse_run(r, i, nrot, nullptr);
    if (run >= 2 && st->sec_a >= 0 && st->real) {
      qf::SparseArgs sa;
      qf::SecBlk sb;
      if (build_sparse(r + i, run, n, false, false, &sa) && to_secblk(sa, n, st->sec_a, st->sec_b, false, &sb)) {
        pend.push_back(sb);
        i += run;
        continue;
      }
    }
    qf_status fs = flush_sector(st, pend);
    if (fs != QF_OK) return fs;
    if (run >= 2) {
      qf::SparseArgs sa;
      if (build_sparse(r + i, run, n, false, false, &sa)) {
        const bool rm = qf::sparse_m_real(sa);
        QF_CUDA(qf::launch_sparse(st->psi, n, st->dt, sa, st->real && rm, st->stream));
        st->real = st->real && rm;
        st->sec_a = st->sec_b = -1;
        i += run;
        continue;
      }
    }
    // greedy tile fusion over consecutive rotations whose X support union stays small
    uint64_t uni = r[i].x;
    size_t j = i + 1;
    while (j < nrot && (int)(j - i) < qf::kTileMaxRot && popc(uni | r[j].x) <= umax) {
      // stop before a run that can become a sparse block
      if (j + 1 < nrot && r[j].x != 0 && r[j + 1].x == r[j].x && r[j].x != r[j - 1].x) break;
      uni |= r[j].x;
      ++j;
    }
    if (j - i >= 2 && n >= 4) {
      qf::TileArgs ta;
      build_tile(st, r, i, j, uni, &ta);
      QF_CUDA(qf::launch_tile(st->psi, n, st->dt, ta, st->stream));
      for (size_t k = i; k < j; ++k) st->real = st->real && keeps_real(r[k].x, r[k].z);
      st->sec_a = st->sec_b = -1;
      i = j;
    } else {
      qf::RotArgs a = rot_args(st->dt, &st->scale, r[i].x, r[i].z, r[i].th);
      QF_CUDA(qf::launch_rot(st->psi, n, st->dt, a, st->stream));
      st->real = st->real && keeps_real(r[i].x, r[i].z);
      if (r[i].x != 0) st->sec_a = st->sec_b = -1;  // a diagonal rotation keeps every occupation
      ++i;
    }
  }
  return flush_sector(st, pend);
}

}  // namespace

extern "C" {

const char* qf_last_error(void) { return t_err.c_str(); }

qf_status qf_state_create(int n, qf_dtype dtype, void* stream, void* dev_buf, size_t dev_buf_bytes,
                          qf_state** out) {
  if (!out) return fail(QF_EINVAL, "out is NULL");
  if (n < 1 || n > QF_MAX_QUBITS) return fail(QF_EINVAL, "qubit count outside 1..QF_MAX_QUBITS");
  if (dtype != QF_C128 && dtype != QF_C64) return fail(QF_EINVAL, "unknown dtype");
  qf_state* st = new qf_state();
  st->n = n;
  st->dt = dtype;
  st->stream = static_cast<cudaStream_t>(stream);
  if (dev_buf) {
    if (dev_buf_bytes < st->bytes() || (reinterpret_cast<uintptr_t>(dev_buf) & 255u)) {
      delete st;
      return fail(QF_EINVAL, "dev_buf too small or not 256-byte aligned");
    }
    st->psi = dev_buf;
  } else {
    if (cudaMalloc(&st->psi, st->bytes()) != cudaSuccess) {
      cudaGetLastError();
      delete st;
      return fail(QF_ENOMEM, "cudaMalloc(state) failed");
    }
    st->own_psi = true;
  }
  if (cudaMalloc(&st->d_partials, kPartials * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&st->d_counter, sizeof(unsigned)) != cudaSuccess) {
    cudaGetLastError();
    if (st->own_psi) cudaFree(st->psi);
    cudaFree(st->d_partials);
    delete st;
    return fail(QF_ENOMEM, "cudaMalloc(scratch) failed");
  }
  if (ensure_out(st, 64) != QF_OK) {
    if (st->own_psi) cudaFree(st->psi);
    cudaFree(st->d_partials);
    cudaFree(st->d_counter);
    delete st;
    return QF_ENOMEM;
  }
  cudaError_t e = cudaMemsetAsync(st->d_counter, 0, sizeof(unsigned), st->stream);
  if (e == cudaSuccess) e = qf::launch_zero_and_set(st->psi, n, dtype, 0ull, st->stream);
  if (e != cudaSuccess) {
    qf_state_destroy(st);
    return fail(QF_ECUDA, std::string("state init: ") + cudaGetErrorString(e));
  }
  *out = st;
  return QF_OK;
}

qf_status qf_state_destroy(qf_state* st) {
  if (!st) return fail(QF_EINVAL, "state is NULL");
  cudaStreamSynchronize(st->stream);
  for (auto& kv : st->plans) free_plan(kv.second);
  if (st->own_psi) cudaFree(st->psi);
  cudaFree(st->lam);
  cudaFree(st->split);
  cudaFree(st->d_secblk);
  cudaFree(st->d_sec_partial);
  cudaFree(st->d_bar);
  cudaFree(st->d_rank);
  cudaFree(st->d_cstate);
  cudaFree(st->d_runblk);
  cudaFree(st->d_log);
  cudaFree(st->d_map);
  cudaFree(st->d_idx);
  cudaFree(st->d_poolblk);
  cudaFree(st->d_small);
  cudaFree(st->d_scoef);
  cudaFree(st->d_sout);
  cudaFreeHost(st->h_scoef);
  cudaFreeHost(st->h_sout);
  cudaFree(st->d_partials);
  cudaFree(st->d_counter);
  cudaFree(st->d_out);
  cudaFreeHost(st->h_out);
  delete st;
  return QF_OK;
}

qf_status qf_set_basis(qf_state* st, uint64_t det) {
  if (!st) return fail(QF_EINVAL, "state is NULL");
  if (st->n < 64 && (det >> st->n)) return fail(QF_EINVAL, "determinant has a bit at or above the qubit count");
  st->scale = 1.0;
  st->real = true;
  st->sec_a = popc(det & kEvenMask);
  st->sec_b = popc(det & ~kEvenMask);
  QF_CUDA(qf::launch_zero_and_set(st->psi, st->n, st->dt, det, st->stream));
  return QF_OK;
}

qf_status qf_apply_pauli_exp(qf_state* st, uint64_t x, uint64_t z, double theta) {
  if (!st) return fail(QF_EINVAL, "state is NULL");
  qf_status v = validate_masks(st, x, z);
  if (v != QF_OK) return v;
  if (!std::isfinite(theta)) return fail(QF_EINVAL, "theta is not finite");
  qf::RotArgs a = rot_args(st->dt, &st->scale, x, z, theta);
  QF_CUDA(qf::launch_rot(st->psi, st->n, st->dt, a, st->stream));
  st->real = st->real && keeps_real(x, z);
  if (x != 0) st->sec_a = st->sec_b = -1;
  return QF_OK;
}

qf_status qf_apply_circuit(qf_state* st, const qf_rot* rots, size_t n_rot) {
  if (!st) return fail(QF_EINVAL, "state is NULL");
  if (n_rot == 0) return QF_OK;
  if (!rots) return fail(QF_EINVAL, "rotation list is NULL");
  std::vector<RotIn> r(n_rot);
  for (size_t k = 0; k < n_rot; ++k) {
    qf_status v = validate_masks(st, rots[k].x, rots[k].z);
    if (v != QF_OK) return v;
    if (!std::isfinite(rots[k].theta)) return fail(QF_EINVAL, "theta is not finite");
    r[k] = RotIn{rots[k].x, rots[k].z, rots[k].theta, 1.0};
  }
  return apply_rotations(st, r.data(), n_rot);
}

qf_status qf_trotter(qf_state* st, const qf_term* terms, size_t n_terms, double time, int steps) {
  if (!st) return fail(QF_EINVAL, "state is NULL");
  if (steps < 1) return fail(QF_EINVAL, "Trotter step count must be at least 1");
  if (!std::isfinite(time)) return fail(QF_EINVAL, "time is not finite");
  if (n_terms == 0) return QF_OK;
  if (!terms) return fail(QF_EINVAL, "term list is NULL");
  std::vector<RotIn> r(n_terms);
  for (size_t k = 0; k < n_terms; ++k) {
    qf_status v = validate_masks(st, terms[k].x, terms[k].z);
    if (v != QF_OK) return v;
    const double th = terms[k].coeff * time / steps;
    if (!std::isfinite(th)) return fail(QF_EINVAL, "coefficient is not finite");
    r[k] = RotIn{terms[k].x, terms[k].z, th, 1.0};
  }
  for (int s = 0; s < steps; ++s) {
    qf_status a = apply_rotations(st, r.data(), n_terms);
    if (a != QF_OK) return a;
  }
  return QF_OK;
}

qf_status qf_expectation(qf_state* st, const qf_term* terms, size_t n_terms, double* re, double* im) {
  if (!st || !re) return fail(QF_EINVAL, "NULL argument");
  if (n_terms && !terms) return fail(QF_EINVAL, "term list is NULL");
  if (im) *im = 0.0;
  if (n_terms == 0) {
    *re = 0.0;
    return QF_OK;
  }
  trim_plans(st);
  const ExpPlan* p = nullptr;
  qf_status ps = get_plan(st, terms, n_terms, &p);
  if (ps != QF_OK) return ps;
  const int nb = qf::reduce_blocks(st->n, st->dt);
  if (st->sec_a >= 0 && st->n <= 2 * qf::kSecMaxPos) {
    // every nonzero amplitude is in one (alpha, beta) sector: sum over its members only
    const qf::SecSpace sp = sector_space(st->n, st->sec_a, st->sec_b);
    QF_CUDA(qf::launch_sector_hpsi(st->psi, nullptr, st->dt, st->real && !p->has_odd, sp, p->rk,
                                   p->d_seclarge, p->nseclarge, p->d_hchunks, st->d_partials, st->d_counter,
                                   st->d_out, kPartials / 2, qf::SecCompact{}, st->stream));
  } else {
    QF_CUDA(qf::launch_expect(st->psi, st->n, st->dt, p->d_groups, p->ngroups, p->d_echunks, st->d_partials,
                              st->d_counter, st->d_out, nb, st->stream));
  }
  QF_CUDA(d2h(st->h_out, st->d_out, sizeof(double), st->stream));
  QF_CUDA(cudaStreamSynchronize(st->stream));
  *re = st->h_out[0] * st->scale * st->scale;
  return QF_OK;
}

// Block structure of a rotation list: runs of same-X, same-parameter, mutually
// commuting rotations become sparse composite blocks (their active rows do not
// depend on the angles, so the structure is kept and only M is refilled);
// anything else is walked rotation by rotation.
std::vector<qf_state::Blk> plan_blocks(const RotIn* r, const int32_t* par, size_t n_rot, int n) {
  using Blk = qf_state::Blk;
  // candidate runs (assuming every run becomes a block), built in parallel
  std::vector<std::pair<size_t, int>> runs;
  for (size_t i = 0; i < n_rot;) {
    const int run = sparse_run(r, i, n_rot, par);
    runs.emplace_back(i, run);
    i += run;
  }
  std::vector<Blk> cand(runs.size());
  std::vector<char> ok(runs.size(), 0);
  qf::HostPool::get().parallel_for(runs.size(), 16, [&](size_t k) {
    const size_t i = runs[k].first;
    const int run = runs[k].second;
    Blk& b = cand[k];
    b.i = i;
    b.j = i + run;
    b.sparse = run >= 2 && build_sparse(r + i, run, n, false, true, &b.fwd) &&
               build_sparse(r + i, run, n, true, true, &b.inv) && b.fwd.nr == b.inv.nr;
    ok[k] = b.sparse;
  });
  // every run a sparse block (a UCC ansatz): the candidates are the plan (a
  // block carries two composites of about 8 KB each; copying them dominated)
  if (std::all_of(ok.begin(), ok.end(), [](char v) { return v != 0; })) return cand;
  // assemble in order; a run that is not a sparse block is walked rotation by rotation
  std::vector<Blk> bl;
  bl.reserve(runs.size());
  for (size_t k = 0; k < runs.size(); ++k) {
    if (ok[k]) {
      bl.push_back(cand[k]);
      continue;
    }
    for (size_t i = runs[k].first; i < runs[k].first + runs[k].second;) {
      const int run = sparse_run(r, i, runs[k].first + runs[k].second, par);
      Blk b;
      b.i = i;
      b.sparse = false;
      if (run >= 2 && build_sparse(r + i, run, n, false, true, &b.fwd) &&
          build_sparse(r + i, run, n, true, true, &b.inv) && b.fwd.nr == b.inv.nr) {
        b.sparse = true;
        b.j = i + run;
      } else {
        b.j = i + 1;
      }
      bl.push_back(b);
      i = b.j;
    }
  }
  return bl;
}

// The lambda buffer, allocated on first need and kept with the handle.
static qf_status ensure_lam(qf_state* st) {
  if (!st->lam && cudaMalloc(&st->lam, st->bytes()) != cudaSuccess) {
    cudaGetLastError();
    st->lam = nullptr;
    return fail(QF_ENOMEM, "cudaMalloc(lambda) failed");
  }
  return QF_OK;
}

// Energy, gradient (grad may be NULL) and, for n_dets basis indices, the
// residuals <b|U^dagger H U|det> / |psi| as (re, im) pairs in res.
// With a pool (n_pool_rot rotations at zero angle, parameters in [0, n_pool)):
// its gradients (Eq. 21) into pool_grad on the compact sector path; when that
// path cannot take the pool, *pool_fallback is set before any GPU work and the
// caller evaluates the pool another way.
static qf_status energy_grad_impl(qf_state* st, uint64_t det, const qf_arot* ansatz, size_t n_rot, const double* t,
                                  size_t n_par, const qf_term* terms, size_t n_terms, double* energy, double* grad,
                                  const uint64_t* dets, size_t n_dets, double* res, const qf_arot* pool = nullptr,
                                  size_t n_pool_rot = 0, size_t n_pool = 0, double* pool_grad = nullptr,
                                  bool* pool_fallback = nullptr) {
  if (!st || !energy) return fail(QF_EINVAL, "NULL argument");
  if ((n_rot && !ansatz) || (n_par && !t) || (n_terms && !terms) || (n_dets && (!dets || !res)))
    return fail(QF_EINVAL, "NULL array");
  for (size_t k = 0; k < n_dets; ++k)
    if (st->n < 64 && (dets[k] >> st->n)) return fail(QF_EINVAL, "residual determinant has a bit at or above the qubit count");
  trim_plans(st);
  const bool want_pool = pool_fallback != nullptr;
  if (want_pool) {
    *pool_fallback = false;
    if ((n_pool_rot && !pool) || (n_pool && !pool_grad)) return fail(QF_EINVAL, "NULL array");
    for (size_t k = 0; k < n_pool_rot; ++k) {
      qf_status v = validate_masks(st, pool[k].x, pool[k].z);
      if (v != QF_OK) return v;
      if (pool[k].param < 0 || (size_t)pool[k].param >= n_pool)
        return fail(QF_EINVAL, "pool parameter index out of range");
      if (!std::isfinite(pool[k].coeff)) return fail(QF_EINVAL, "pool coefficient is not finite");
    }
  }
  if (st->n < 64 && (det >> st->n)) return fail(QF_EINVAL, "determinant has a bit at or above the qubit count");
  // block structure: sparse composite blocks (same X, same parameter, commuting) or single rotations
  using Blk = qf_state::Blk;
  // the last ansatz plan first (one comparison, no hashing), then by content key
  uint64_t akey = st->last_ansatz_key;
  auto ait = st->ansatz_plans.find(akey);
  if (ait == st->ansatz_plans.end() || !same_arots(ait->second.src, ansatz, n_rot)) {
    akey = content_key(ansatz, n_rot * sizeof(qf_arot), 0x13198A2E03707344ull ^ (uint64_t)st->n);
    ait = st->ansatz_plans.find(akey);
    if (ait != st->ansatz_plans.end() && !same_arots(ait->second.src, ansatz, n_rot)) {
      // another rotation list with the same key: the key only picks the slot
      st->ansatz_plans.erase(ait);
      ait = st->ansatz_plans.end();
      st->parts_key = 0;
      st->map_key = 0;
    }
  }
  // a cached plan's rotations had their masks checked when it was built
  const bool known = ait != st->ansatz_plans.end();
  std::vector<RotIn> r(n_rot);
  std::vector<int32_t> par(n_rot);
  for (size_t k = 0; k < n_rot; ++k) {
    if (!known) {
      qf_status v = validate_masks(st, ansatz[k].x, ansatz[k].z);
      if (v != QF_OK) return v;
    }
    if (ansatz[k].param < 0 || (size_t)ansatz[k].param >= n_par)
      return fail(QF_EINVAL, "ansatz parameter index out of range");
    const double th = ansatz[k].coeff * t[ansatz[k].param];
    if (!std::isfinite(th)) return fail(QF_EINVAL, "theta is not finite");
    r[k] = RotIn{ansatz[k].x, ansatz[k].z, th, ansatz[k].coeff};
    par[k] = ansatz[k].param;
  }
  st->last_ansatz_key = akey;
  if (ait == st->ansatz_plans.end()) {
    // first sight of this ansatz: find its block structure
    std::vector<Blk> bl = plan_blocks(r.data(), par.data(), n_rot, st->n);
    qf_state::AnsatzPlan plan;
    plan.src.assign(ansatz, ansatz + n_rot);
    plan.blocks = std::move(bl);
    ait = st->ansatz_plans.emplace(akey, std::move(plan)).first;
  }
  ait->second.last_use = st->calls;
  qf_state::AnsatzPlan& ap = ait->second;
  std::vector<Blk>& blocks = ap.blocks;
  const size_t nblk = blocks.size();
  qf_status os = ensure_out(st, nblk + 2 + 2 * n_dets);
  if (os != QF_OK) return os;
  const bool need_reverse = !want_pool || grad || n_dets;
  const ExpPlan* p = nullptr;
  if (n_terms) {
    qf_status ps = get_plan(st, terms, n_terms, &p);
    if (ps != QF_OK) return ps;
  }
  const int n = st->n;
  const int na = popc(det & kEvenMask), nbeta = popc(det & ~kEvenMask);
  const bool lreal = !p || !p->has_odd;
  // part-local runs: parts of at most kRunPartTarget members (and what shared memory holds)
  const uint64_t cap = std::min<uint64_t>(
      kRunPartTarget, std::min(qf::sector_run_capacity(st->dt, false, true, false),
                               qf::sector_run_capacity(st->dt, true, lreal, false)));
  const bool sec_cached =
      ap.sec_ok && ap.sec_n == n && ap.sec_na == na && ap.sec_nb == nbeta && ap.sec_cap == cap;
  // new angles: refill every block's composites (and, with a cached run plan, its
  // sector form), spread over the host pool
  std::atomic<bool> sec_good(true);
  // (a fresh plan's composites are refilled too, so that the first call and
  // every later call with the same angles give bit-identical results)
  {
    qf::HostPool::get().parallel_for(nblk, 32, [&](size_t k) {
      Blk& b = blocks[k];
      if (!b.sparse) return;
      refill_sparse(&r[b.i], (int)(b.j - b.i), false, &b.fwd);
      if (!adjoint_composite(b.fwd, &b.inv)) refill_sparse(&r[b.i], (int)(b.j - b.i), true, &b.inv);
      if (sec_cached) {
        qf::RunBlk& F = ap.runs.blks[k];
        qf::RunBlk& I = ap.runs.blks[nblk + k];
        if (!sector_mq(b.fwd, false, F.m, F.q) || !sector_mq(b.inv, true, I.m, I.q)) sec_good = false;
        qf::runblk_f32(F);
        qf::runblk_f32(I);
      }
    });
  }
  // Sector path: every block is a two-row excitation that keeps the reference's
  // numbers of occupied even and odd qubits, so the whole evaluation runs on the
  // members of that sector, stored contiguously (compact layout) in a buffer of
  // the handle; psi itself is only reset to |det> at the end.
  bool sector = !blocks.empty() && n <= 2 * qf::kSecMaxPos;
  // residuals outside the sector need H psi off the sector too: general path
  for (size_t k = 0; sector && k < n_dets; ++k)
    sector = popc(dets[k] & kEvenMask) == na && popc(dets[k] & ~kEvenMask) == nbeta;
  if (sector && !sec_cached) {
    // first evaluation of this ansatz in this sector: the run plan
    std::vector<qf::SecBlk> sec(2 * nblk);
    for (size_t bi = 0; sector && bi < nblk; ++bi)
      sector = blocks[bi].sparse && to_secblk(blocks[bi].fwd, n, na, nbeta, false, &sec[bi]) &&
               to_secblk(blocks[bi].inv, n, na, nbeta, true, &sec[nblk + bi]);
    ap.sec_ok = sector && build_runs(sec.data(), nblk, n, na, nbeta, cap, &ap.runs);
    ap.sec_n = n;
    ap.sec_na = na;
    ap.sec_nb = nbeta;
    ap.sec_cap = cap;
    st->parts_key = 0;
    sector = ap.sec_ok;
  } else if (sector) {
    sector = sec_good.load();  // a block that lost the sector form this time: general path
  }
  if (sector) {
    st->scale = 1.0;
    st->real = true;
    st->sec_a = na;
    st->sec_b = nbeta;
    if (!p) {  // no Hamiltonian terms: E = 0, a zero gradient and zero residuals
      QF_CUDA(qf::launch_zero_and_set(st->psi, n, st->dt, det, st->stream));
      QF_CUDA(cudaStreamSynchronize(st->stream));
      *energy = 0.0;
      if (grad)
        for (size_t k = 0; k < n_par; ++k) grad[k] = 0.0;
      for (size_t k = 0; k < 2 * n_dets; ++k) res[k] = 0.0;
      for (size_t k = 0; k < n_pool; ++k) pool_grad[k] = 0.0;
      return QF_OK;
    }
    // the pool (its blocks at zero angle) as sector blocks, planned once per handle
    qf_state::AnsatzPlan* pp = nullptr;
    uint64_t pkey0 = 0;  // the pool's content key
    if (want_pool) {
      if (!lreal) {  // overlaps on the packed (psi, lambda) need a real lambda
        *pool_fallback = true;
        return QF_OK;
      }
      pkey0 = content_key(pool, n_pool_rot * sizeof(qf_arot), 0x452821E638D01377ull ^ (uint64_t)n);
      auto pit = st->ansatz_plans.find(pkey0);
      if (pit != st->ansatz_plans.end() && (&pit->second == &ap || !same_arots(pit->second.src, pool, n_pool_rot))) {
        if (&pit->second == &ap) return fail(QF_EINVAL, "pool and ansatz plans share a cache key");
        st->ansatz_plans.erase(pit);
        pit = st->ansatz_plans.end();
        st->pool_key = 0;
      }
      if (pit == st->ansatz_plans.end()) {
        std::vector<RotIn> rp(n_pool_rot);
        std::vector<int32_t> ppar(n_pool_rot);
        for (size_t k = 0; k < n_pool_rot; ++k) {
          rp[k] = RotIn{pool[k].x, pool[k].z, 0.0, pool[k].coeff};
          ppar[k] = pool[k].param;
        }
        qf_state::AnsatzPlan plan;
        plan.src.assign(pool, pool + n_pool_rot);
        plan.blocks = plan_blocks(rp.data(), ppar.data(), n_pool_rot, n);
        pit = st->ansatz_plans.emplace(pkey0, std::move(plan)).first;
      }
      pit->second.last_use = st->calls;
      pp = &pit->second;
      if (!(pp->sec_ok && pp->sec_n == n && pp->sec_na == na && pp->sec_nb == nbeta && pp->sec_cap == cap)) {
        const size_t nbp = pp->blocks.size();
        std::vector<qf::SecBlk> sec(2 * nbp);
        bool ok = nbp > 0;
        for (size_t bi = 0; ok && bi < nbp; ++bi)
          ok = pp->blocks[bi].sparse && to_secblk(pp->blocks[bi].fwd, n, na, nbeta, false, &sec[bi]) &&
               to_secblk(pp->blocks[bi].inv, n, na, nbeta, true, &sec[nbp + bi]);
        pp->sec_ok = ok && build_runs(sec.data(), nbp, n, na, nbeta, cap, &pp->runs);
        pp->sec_n = n;
        pp->sec_na = na;
        pp->sec_nb = nbeta;
        pp->sec_cap = cap;
        st->pool_key = 0;
      }
      if (!pp->sec_ok) {
        *pool_fallback = true;
        return QF_OK;
      }
      const size_t nbp = pp->blocks.size();
      qf_status po = ensure_out(st, nblk + 2 + 2 * n_dets + nbp);
      if (po != QF_OK) return po;
    }
    const SectorRuns& rs = ap.runs;
    // a real state with a Hamiltonian of molecular form takes the direct tables
    // (built before this call queues any kernel: their upload synchronises the stream)
    ExpPlan* pm = const_cast<ExpPlan*>(p);
    if (lreal && st->n <= 32) {
      qf_status ds = ensure_direct(st, pm);
      if (ds != QF_OK) return ds;
    }
    const qf::SecSpace sp = sector_space(n, na, nbeta);
    qf::SecCompact cm{};
    qf_status cs = ensure_compact(st, sp, na, nbeta, &cm);
    if (cs != QF_OK) return cs;
    size_t partials = nblk * (size_t)rs.pmax;
    if (pp) partials = std::max(partials, pp->blocks.size() * (size_t)pp->runs.pmax);
    qf_status bs = ensure_sector_buffers(st, 1, partials);
    if (bs != QF_OK) return bs;
    const size_t blk_bytes = rs.blks.size() * sizeof(qf::RunBlk);
    const size_t part_bytes = rs.parts.size() * sizeof(qf::RunPart);
    const void* before = st->d_runblk;
    bs = ensure_buf(&st->d_runblk, &st->runblk_cap, blk_bytes + part_bytes + rs.strs.size() * sizeof(uint16_t),
                    "sector run descriptors");
    if (bs != QF_OK) return bs;
    const qf::RunBlk* d_blks = static_cast<const qf::RunBlk*>(st->d_runblk);
    const qf::RunPart* d_parts =
        reinterpret_cast<const qf::RunPart*>(static_cast<const char*>(st->d_runblk) + blk_bytes);
    QF_CUDA(h2d(st->d_runblk, rs.blks.data(), blk_bytes, st->stream));
    // the parts depend only on the plan and the sector: upload them when those change
    const uint64_t pkey = content_key(nullptr, 0, akey ^ ((uint64_t)na << 40) ^ ((uint64_t)nbeta << 48) ^ cap) | 1ull;
    if (st->parts_key != pkey || st->d_runblk != before) {
      QF_CUDA(h2d(static_cast<char*>(st->d_runblk) + blk_bytes, rs.parts.data(), part_bytes, st->stream));
      if (!rs.strs.empty())
        QF_CUDA(h2d(static_cast<char*>(st->d_runblk) + blk_bytes + part_bytes, rs.strs.data(),
                    rs.strs.size() * sizeof(uint16_t), st->stream));
      st->parts_key = pkey;
    }
    const uint64_t members = (uint64_t)sp.cnt_e * sp.cnt_o;
    // a real lambda shares psi's slots (psi real parts, lambda imaginary parts)
    void* cpsi = st->d_cstate;
    void* clam = lreal ? cpsi : static_cast<char*>(cpsi) + members * st->elem();
    // forward log (real lambda only): psi after each block, so that the reverse need
    // not un-rotate psi; up to kLogMaxBytes, else (or when it does not fit) the
    // reverse un-rotates psi
    void* log = nullptr;
    const size_t log_bytes = (size_t)rs.logitems * st->elem();  // one (psi_i0, psi_i1) pair per item
    if (need_reverse && lreal && rs.log_ok && !st->log_failed && log_bytes <= kLogMaxBytes) {
      if (ensure_buf(&st->d_log, &st->log_cap, log_bytes, "sector log") == QF_OK)
        log = st->d_log;
      else
        st->log_failed = true;
    }
    const int nruns = (int)rs.runs.size();
    const uint16_t* d_strs =
        rs.strs.empty() ? nullptr
                        : reinterpret_cast<const uint16_t*>(static_cast<const char*>(st->d_runblk) + blk_bytes +
                                                            part_bytes);
    // item maps of the sweeps, built on the device whenever the parts change
    const uint32_t* d_map = nullptr;
    if (rs.map_ok && rs.mapwords > 0 && rs.mapwords <= kMapMaxWords) {
      const void* mbefore = st->d_map;
      if (ensure_buf(&st->d_map, &st->map_cap, (size_t)rs.mapwords * sizeof(uint32_t), "sweep item maps") == QF_OK) {
        if (st->map_key != pkey || st->d_map != mbefore) {
          QF_CUDA(qf::launch_run_itemmaps(rs.runs.data(), nruns, d_parts, d_blks, cm, d_strs,
                                          static_cast<uint32_t*>(st->d_map), st->stream));
          st->map_key = pkey;
        }
        d_map = static_cast<const uint32_t*>(st->d_map);
      }
    }
    st->run_items = rs.run_items;
    const bool hdirect = lreal && pm->direct == 1;
    // complex128 in QF_HPSI_DS mode: the mapped sweeps run in double-single arithmetic;
    // the reverse must agree with the forward, whose log it reads
    const bool sweep_ds = st->dt == QF_C128 && st->hpsi_mode == QF_HPSI_DS && d_map != nullptr &&
                          (log != nullptr || !need_reverse);
    // and the compact state stays in double-single form from the reset to the end
    // of the reverse when the sweeps, the direct H|psi> and the residual gather are
    // all that touch it (the pool overlaps read FP64 members)
    const bool dss = sweep_ds && hdirect && !pp;
    const uint64_t c0 = compact_of(det, sp);
    if (dss)  // member c0 = (1, 0, 0, 0) as floats: element 2 c0 of 2 * members float pairs
      QF_CUDA(qf::launch_zero_and_set_count(cpsi, 2 * members, QF_C64, 2 * c0, st->stream));
    else
      QF_CUDA(qf::launch_zero_and_set_count(cpsi, members, st->dt, c0, st->stream));
    QF_CUDA(qf::launch_sector_runs(cpsi, nullptr, st->dt, false, true, rs.runs.data(), nruns, d_parts, d_blks,
                                   (int)nblk, nullptr, rs.pmax, nullptr, cm, log, d_strs, d_map, sweep_ds, dss,
                                   st->stream));
    double* d_e = st->d_out + nblk;
    // double-single pair products (complex128, QF_HPSI_DS): the amplitudes' float
    // split sits in the compact buffer's second half, unused by a packed real lambda,
    // followed (double-single state) by psi's FP64 values
    float2* split = (st->dt == QF_C128 && st->hpsi_mode == QF_HPSI_DS)
                        ? reinterpret_cast<float2*>(static_cast<char*>(cpsi) + members * st->elem())
                        : nullptr;
    double* psid = split ? reinterpret_cast<double*>(split + members) : nullptr;
    if (hdirect)
      QF_CUDA(qf::launch_sector_hpsi_direct(cpsi, st->dt, sp, pm->dtab, cm, st->d_partials, st->d_counter, d_e,
                                            kPartials / 2, split, psid, dss, st->stream));
    else
      QF_CUDA(qf::launch_sector_hpsi(cpsi, clam, st->dt, lreal, sp, p->rk, p->d_seclarge, p->nseclarge,
                                     p->d_hchunks, st->d_partials, st->d_counter, d_e, kPartials / 2, cm,
                                     st->stream));
    const size_t npool_blk = pp ? pp->blocks.size() : 0;
    double* d_pool = st->d_out + nblk + 2 + 2 * n_dets;
    if (pp) {  // every pool operator's overlap with the final (psi, lambda): nothing rotated
      const SectorRuns& pr = pp->runs;
      const size_t pblk = pr.blks.size() * sizeof(qf::RunBlk), ppart = pr.parts.size() * sizeof(qf::RunPart);
      const void* pbefore = st->d_poolblk;
      bs = ensure_buf(&st->d_poolblk, &st->poolblk_cap, pblk + ppart + pr.strs.size() * sizeof(uint16_t),
                      "pool run descriptors");
      if (bs != QF_OK) return bs;
      const uint64_t key =
          content_key(nullptr, 0, pkey0 ^ ((uint64_t)na << 40) ^ ((uint64_t)nbeta << 48) ^ cap) | 1ull;
      if (st->pool_key != key || st->d_poolblk != pbefore) {  // zero angle: the descriptors never change
        char* base = static_cast<char*>(st->d_poolblk);
        QF_CUDA(h2d(base, pr.blks.data(), pblk, st->stream));
        QF_CUDA(h2d(base + pblk, pr.parts.data(), ppart, st->stream));
        if (!pr.strs.empty()) QF_CUDA(h2d(base + pblk + ppart, pr.strs.data(), pr.strs.size() * 2, st->stream));
        st->pool_key = key;
      }
      const char* base = static_cast<const char*>(st->d_poolblk);
      QF_CUDA(qf::launch_sector_overlaps(
          cpsi, st->dt, pr.runs.data(), (int)pr.runs.size(), reinterpret_cast<const qf::RunPart*>(base + pblk),
          reinterpret_cast<const qf::RunBlk*>(base) + npool_blk, (int)npool_blk, st->d_sec_partial, pr.pmax, d_pool,
          cm, pr.strs.empty() ? nullptr : reinterpret_cast<const uint16_t*>(base + pblk + ppart), st->stream));
    }
    if (need_reverse)
      QF_CUDA(qf::launch_sector_runs(cpsi, clam, st->dt, true, lreal, rs.runs.data(), nruns, d_parts, d_blks + nblk,
                                     (int)nblk, st->d_sec_partial, rs.pmax, st->d_out, cm, log, d_strs, d_map,
                                     sweep_ds, dss, st->stream));
    if (n_dets) {  // residuals: lambda after the reverse sweep is U^dagger H psi
      std::vector<int64_t> idx(n_dets);
      for (size_t k = 0; k < n_dets; ++k) idx[k] = (int64_t)compact_of(dets[k], sp);
      QF_CUDA(gather_residuals(st, lreal ? cpsi : clam, lreal, dss, idx, st->d_out + nblk + 2));
    }
    QF_CUDA(qf::launch_zero_and_set(st->psi, n, st->dt, det, st->stream));
    QF_CUDA(d2h(st->h_out, st->d_out, (nblk + 2 + 2 * n_dets + npool_blk) * sizeof(double), st->stream));
    QF_CUDA(cudaStreamSynchronize(st->stream));
    double nrm = st->h_out[nblk + 1];
    if (!(nrm > 0.0)) nrm = 1.0;
    *energy = st->h_out[nblk] / nrm;
    if (grad) {
      for (size_t k = 0; k < n_par; ++k) grad[k] = 0.0;
      for (size_t bi = 0; bi < nblk; ++bi) grad[par[blocks[bi].i]] += 2.0 * st->h_out[bi] / nrm;
    }
    const double rs_scale = 1.0 / std::sqrt(nrm);  // residuals scale with |psi|
    for (size_t k = 0; k < 2 * n_dets; ++k) res[k] = st->h_out[nblk + 2 + k] * rs_scale;
    if (pp) {
      for (size_t k = 0; k < n_pool; ++k) pool_grad[k] = 0.0;
      for (size_t bi = 0; bi < npool_blk; ++bi)
        pool_grad[pool[pp->blocks[bi].i].param] += 2.0 * st->h_out[nblk + 2 + 2 * n_dets + bi] / nrm;
    }
    return QF_OK;
  }
  if (want_pool) {  // the general path takes no pool
    *pool_fallback = true;
    return QF_OK;
  }
  qf_status ls = ensure_lam(st);
  if (ls != QF_OK) return ls;
  st->scale = 1.0;
  st->real = true;
  st->sec_a = st->sec_b = -1;
  QF_CUDA(qf::launch_zero_and_set(st->psi, n, st->dt, det, st->stream));
  for (const Blk& b : blocks) {
    if (b.sparse) {
      const bool rm = qf::sparse_m_real(b.fwd);
      QF_CUDA(qf::launch_sparse(st->psi, n, st->dt, b.fwd, st->real && rm, st->stream));
      st->real = st->real && rm;
    } else {
      qf::RotArgs a = rot_args(st->dt, &st->scale, r[b.i].x, r[b.i].z, r[b.i].th);
      QF_CUDA(qf::launch_rot(st->psi, n, st->dt, a, st->stream));
      st->real = st->real && keeps_real(r[b.i].x, r[b.i].z);
    }
  }
  const double s_fwd = st->scale;
  const int nb = qf::reduce_blocks(n, st->dt);
  double* d_e = st->d_out + blocks.size();
  const bool hreal = st->real && p && !p->has_odd;
  if (p && n >= 10) {
    qf_status ts = ensure_tiled(st, const_cast<ExpPlan*>(p));
    if (ts != QF_OK) return ts;
  }
  if (p && n >= 12 && hreal && st->dt == QF_C128 && st->hpsi_mode == QF_HPSI_DS) {
    if (!st->split && cudaMalloc(&st->split, sizeof(float2) << n) != cudaSuccess) {
      cudaGetLastError();
      st->split = nullptr;
      return fail(QF_ENOMEM, "cudaMalloc(double-single split) failed");
    }
    QF_CUDA(qf::launch_hpsi_ds(st->psi, st->lam, st->split, n, p->d_classes[2], p->nclasses[2], p->d_hgroups,
                               p->d_wchunks_s, st->d_partials, st->d_counter, d_e, nb, st->stream));
  } else if (p && n >= 10) {
    // tiles of 2^11 amplitudes when the state is real (fewer registers per element), else 2^10
    const int v = (hreal && n >= 11) ? 1 : 0;
    QF_CUDA(qf::launch_hpsi_tiled(st->psi, st->lam, n, st->dt, 10 + v, hreal, p->d_classes[v], p->nclasses[v],
                                  p->d_hgroups, st->dt == QF_C128 ? (const void*)p->d_wchunks
                                                                 : (const void*)p->d_wchunks_f,
                                  st->d_partials, st->d_counter, d_e, nb, st->stream));
  } else if (p) {
    QF_CUDA(qf::launch_hpsi(st->psi, st->lam, n, st->dt, p->d_groups, p->ngroups, p->d_hchunks, st->d_partials,
                            st->d_counter, d_e, nb, st->stream));
  } else {
    QF_CUDA(cudaMemsetAsync(st->lam, 0, st->bytes(), st->stream));
    QF_CUDA(cudaMemsetAsync(d_e, 0, 2 * sizeof(double), st->stream));
  }
  // reverse sweep; psi and lam share one scale
  std::vector<double> s2(blocks.size());
  double sc = s_fwd;
  // psi and lambda = H psi are both real when psi is real and H has no odd-Y term
  bool both_real = st->real && (!p || !p->has_odd);
  for (size_t bi = blocks.size(); bi-- > 0;) {
    const Blk& b = blocks[bi];
    s2[bi] = sc * sc;
    if (b.sparse) {
      const bool rm = qf::sparse_m_real(b.inv);
      QF_CUDA(qf::launch_adj_sparse(st->psi, st->lam, n, st->dt, b.inv, both_real && rm, st->d_partials,
                                    st->d_counter, st->d_out + bi, nb, st->stream));
      both_real = both_real && rm;
    } else {
      qf::RotArgs a = rot_args(st->dt, &sc, r[b.i].x, r[b.i].z, -r[b.i].th);
      QF_CUDA(qf::launch_adj_rot(st->psi, st->lam, n, st->dt, a, st->d_partials, st->d_counter, st->d_out + bi, nb,
                                 st->stream));
      both_real = both_real && keeps_real(r[b.i].x, r[b.i].z);
    }
  }
  st->scale = sc;
  st->real = both_real;
  if (n_dets) {  // residuals: lambda after the reverse sweep is U^dagger H psi (scale sc)
    std::vector<int64_t> idx(dets, dets + n_dets);
    QF_CUDA(gather_residuals(st, st->lam, false, false, idx, st->d_out + blocks.size() + 2));
  }
  QF_CUDA(d2h(st->h_out, st->d_out, (blocks.size() + 2 + 2 * n_dets) * sizeof(double), st->stream));
  QF_CUDA(cudaStreamSynchronize(st->stream));
  // U(t)|det> has unit norm; dividing by the computed <psi|psi> (FP64) removes the
  // rounding drift of the stored norm (the Rayleigh quotient and its gradient;
  // <psi|P_k|psi> is real, so the gradient needs only the same factor).
  double nrm = p ? st->h_out[blocks.size() + 1] * s_fwd * s_fwd : 1.0;
  if (!(nrm > 0.0)) nrm = 1.0;
  *energy = st->h_out[blocks.size()] * s_fwd * s_fwd / nrm;
  if (grad) {
    for (size_t k = 0; k < n_par; ++k) grad[k] = 0.0;
    for (size_t bi = 0; bi < blocks.size(); ++bi) {
      const Blk& b = blocks[bi];
      const double g = 2.0 * st->h_out[bi] * s2[bi] / nrm;
      if (b.sparse)
        grad[par[b.i]] += g;
      else
        grad[par[b.i]] += r[b.i].coeff * g;
    }
  }
  const double rs_scale = sc / std::sqrt(nrm);  // stored lambda times the shared scale, over |psi|
  for (size_t k = 0; k < 2 * n_dets; ++k) res[k] = st->h_out[blocks.size() + 2 + k] * rs_scale;
  return QF_OK;
}

qf_status qf_energy_grad(qf_state* st, uint64_t det, const qf_arot* ansatz, size_t n_rot, const double* t,
                         size_t n_par, const qf_term* terms, size_t n_terms, double* energy, double* grad) {
  if (n_par && !grad) return fail(QF_EINVAL, "NULL array");
  return energy_grad_impl(st, det, ansatz, n_rot, t, n_par, terms, n_terms, energy, grad, nullptr, 0, nullptr);
}

namespace {

qf_status ensure_host(void** p, size_t* cap, size_t bytes, const char* what) {
  if (bytes <= *cap) return QF_OK;
  cudaFreeHost(*p);
  *p = nullptr;
  *cap = 0;
  if (cudaMallocHost(p, bytes) != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return fail(QF_ENOMEM, std::string("cudaMallocHost(") + what + ") failed");
  }
  *cap = bytes;
  return QF_OK;
}

// Requests r0 .. n_req - 1 of qf_energy_grad_multi in one launch (qf::SmallEval),
// when the handle's cached plans allow it: the ansatz and the Hamiltonian planned
// before for this sector, every block a real two-row sector block, the direct
// H|psi> tables, and a sector small enough for one CTA's shared memory.
// Otherwise returns QF_OK with *done = false and touches nothing.
qf_status multi_small(qf_state* st, uint64_t det, const qf_arot* ansatz, size_t n_rot, const double* t,
                      size_t n_par, size_t r0, size_t n_req, const qf_term* terms, size_t n_terms,
                      double* energies, double* grads, bool* done) {
  *done = false;
  const int n = st->n;
  if (n > 32 || n_terms == 0 || n_rot == 0 || r0 >= n_req) return QF_OK;
  auto ait = st->ansatz_plans.find(st->last_ansatz_key);
  if (ait == st->ansatz_plans.end() || !same_arots(ait->second.src, ansatz, n_rot)) {
    ait = st->ansatz_plans.find(content_key(ansatz, n_rot * sizeof(qf_arot), 0x13198A2E03707344ull ^ (uint64_t)n));
    if (ait == st->ansatz_plans.end() || !same_arots(ait->second.src, ansatz, n_rot)) return QF_OK;
  }
  auto same_terms = [&](const std::vector<qf_term>& seen) {
    return seen.size() == n_terms && std::memcmp(seen.data(), terms, n_terms * sizeof(qf_term)) == 0;
  };
  auto pit = st->plans.find(st->last_plan_key);
  if (pit == st->plans.end() || !same_terms(pit->second.terms)) {
    pit = st->plans.find(content_key(terms, n_terms * sizeof(qf_term), 0x243F6A8885A308D3ull ^ (uint64_t)n));
    if (pit == st->plans.end() || !same_terms(pit->second.terms)) return QF_OK;
  }
  qf_state::AnsatzPlan& ap = ait->second;
  ExpPlan& hp = pit->second;
  if (hp.has_odd || hp.direct != 1) return QF_OK;
  const int na = popc(det & kEvenMask), nbeta = popc(det & ~kEvenMask);
  const uint64_t cap = std::min<uint64_t>(
      kRunPartTarget, std::min(qf::sector_run_capacity(st->dt, false, true, false),
                               qf::sector_run_capacity(st->dt, true, true, false)));
  if (!(ap.sec_ok && ap.sec_n == n && ap.sec_na == na && ap.sec_nb == nbeta && ap.sec_cap == cap)) return QF_OK;
  const qf::SecSpace sp = sector_space(n, na, nbeta);
  const uint32_t members = sp.cnt_e * sp.cnt_o;
  if (qf::small_eval_smem(st->dt, members, sp.ko, sp.no) == 0) return QF_OK;
  const std::vector<qf_state::Blk>& blocks = ap.blocks;
  const size_t nblk = blocks.size();
  for (const auto& b : blocks) {  // the reverse reads the forward geometry with the inverse's coefficients
    if (!b.sparse || b.fwd.nr != 2 || b.inv.nr != 2 || b.fwd.nzc != b.inv.nzc) return QF_OK;
    if (b.fwd.pat[0] != b.inv.pat[0] || b.fwd.pat[1] != b.inv.pat[1]) return QF_OK;
    for (int j = 0; j < b.fwd.nzc; ++j)
      if (b.fwd.zc[j] != b.inv.zc[j]) return QF_OK;
  }
  // parameters: indices and angles of every request
  for (size_t k = 0; k < n_rot; ++k)
    if (ansatz[k].param < 0 || (size_t)ansatz[k].param >= n_par)
      return fail(QF_EINVAL, "ansatz parameter index out of range");
  for (size_t q = r0; q < n_req; ++q)
    for (size_t k = 0; k < n_rot; ++k)
      if (!std::isfinite(ansatz[k].coeff * t[q * n_par + ansatz[k].param]))
        return fail(QF_EINVAL, "theta is not finite");
  // the forward blocks' geometry for this sector, on the device once
  const uint64_t skey = content_key(nullptr, 0, ait->first ^ ((uint64_t)na << 40) ^ ((uint64_t)nbeta << 48)) | 1ull;
  if (st->small_key != skey) {
    std::vector<qf::SecBlk> g(nblk);
    for (size_t b = 0; b < nblk; ++b)
      if (!to_secblk(blocks[b].fwd, n, na, nbeta, false, &g[b])) return QF_OK;
    qf_status bs = ensure_buf(&st->d_small, &st->small_cap, nblk * sizeof(qf::SecBlk), "small-request blocks");
    if (bs != QF_OK) return bs;
    QF_CUDA(h2d(st->d_small, g.data(), nblk * sizeof(qf::SecBlk), st->stream));
    QF_CUDA(cudaStreamSynchronize(st->stream));  // g is freed on return
    st->small_key = skey;
  }
  qf::SecCompact cm{};
  qf_status cs = ensure_compact(st, sp, na, nbeta, &cm);
  if (cs != QF_OK) return cs;
  ap.last_use = hp.last_use = st->calls;
  st->last_ansatz_key = ait->first;
  st->last_plan_key = pit->first;
  // per request and block: the forward composite minus I, its transpose (the
  // inverse's, the composite being real orthogonal), and the inverse's generator
  // entry q01 (angle independent), in the state's real type
  const size_t nr = n_req - r0;
  const bool c128 = st->dt == QF_C128;
  const size_t rec = (size_t)qf::kSmallCoef * (c128 ? sizeof(double) : sizeof(float));
  qf_status hs = ensure_host(&st->h_scoef, &st->h_scoef_cap, nr * nblk * rec, "small-request coefficients");
  if (hs != QF_OK) return hs;
  std::atomic<bool> real(true);
  qf::HostPool::get().parallel_for(nr * nblk, 64, [&](size_t k) {
    const size_t q = k / nblk, b = k - q * nblk;
    const qf_state::Blk& B = blocks[b];
    const double* tq = t + (r0 + q) * n_par;
    const int len = (int)(B.j - B.i);
    RotIn rb_buf[16];
    std::vector<RotIn> rb_heap;
    RotIn* rr = rb_buf;
    if (len > 16) {
      rb_heap.resize(len);
      rr = rb_heap.data();
    }
    for (int u = 0; u < len; ++u) {
      const qf_arot& a = ansatz[B.i + u];
      rr[u] = RotIn{a.x, a.z, a.coeff * tq[a.param], a.coeff};
    }
    double m[4][2][2] = {};
    bool ok = true;
    compose_sparse(rr, len, false, B.fwd, [&](int c, int i, int j, cplx d) {
      m[c][i][j] = d.real();
      if (d.imag() != 0.0) ok = false;
    });
    double mi[4][2][2], qi[4][2][2];
    if (!sector_mq(B.inv, true, mi, qi)) ok = false;
    if (!ok) real = false;
    const int ncls = 1 << B.fwd.nzc;
    double v[qf::kSmallCoef];
    for (int c = 0; c < 4; ++c) {
      const int cc = c < ncls ? c : 0;
      for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j) {
          v[4 * c + 2 * i + j] = m[cc][i][j];
          v[16 + 4 * c + 2 * i + j] = m[cc][j][i];
        }
      v[32 + c] = qi[c][0][1];
    }
    unsigned char* dst = static_cast<unsigned char*>(st->h_scoef) + k * rec;
    if (c128) {
      std::memcpy(dst, v, sizeof(v));
    } else {
      float f[qf::kSmallCoef];
      for (int u = 0; u < qf::kSmallCoef; ++u) f[u] = (float)v[u];
      std::memcpy(dst, f, sizeof(f));
    }
  });
  if (!real.load()) return QF_OK;
  const size_t outn = nr * (nblk + 2);
  qf_status bs = ensure_buf(&st->d_scoef, &st->scoef_cap, nr * nblk * rec, "small-request coefficients");
  if (bs == QF_OK) bs = ensure_buf(&st->d_sout, &st->sout_cap, outn * sizeof(double), "small-request results");
  if (bs == QF_OK) bs = ensure_host(&st->h_sout, &st->h_sout_cap, outn * sizeof(double), "small-request results");
  if (bs != QF_OK) return bs;
  QF_CUDA(h2d(st->d_scoef, st->h_scoef, nr * nblk * rec, st->stream));
  qf::SmallEval a{};
  a.blks = static_cast<const qf::SecBlk*>(st->d_small);
  a.nblk = (int)nblk;
  a.coef = st->d_scoef;
  a.d = hp.dtab;
  a.cnt_e = sp.cnt_e;
  a.cnt_o = sp.cnt_o;
  a.ke = sp.ke;
  a.ko = sp.ko;
  a.ra = cm.ra;
  a.rb = cm.rb;
  a.c0 = (uint32_t)compact_of(det, sp);
  a.out = static_cast<double*>(st->d_sout);
  QF_CUDA(qf::launch_small_eval(a, st->dt, (int)nr, st->stream));
  st->scale = 1.0;
  st->real = true;
  st->sec_a = na;
  st->sec_b = nbeta;
  QF_CUDA(qf::launch_zero_and_set(st->psi, n, st->dt, det, st->stream));
  QF_CUDA(d2h(st->h_sout, st->d_sout, outn * sizeof(double), st->stream));
  QF_CUDA(cudaStreamSynchronize(st->stream));
  const double* ho = static_cast<const double*>(st->h_sout);
  for (size_t q = 0; q < nr; ++q) {
    const double* o = ho + q * (nblk + 2);
    double nrm = o[nblk + 1];
    if (!(nrm > 0.0)) nrm = 1.0;
    energies[r0 + q] = o[nblk] / nrm;
    if (grads) {
      double* gq = grads + (r0 + q) * n_par;
      for (size_t k = 0; k < n_par; ++k) gq[k] = 0.0;
      for (size_t b = 0; b < nblk; ++b) gq[ansatz[blocks[b].i].param] += 2.0 * o[b] / nrm;
    }
  }
  *done = true;
  return QF_OK;
}

}  // namespace

qf_status qf_energy_grad_multi(qf_state* st, uint64_t det, const qf_arot* ansatz, size_t n_rot, const double* t,
                               size_t n_par, size_t n_req, const qf_term* terms, size_t n_terms, double* energies,
                               double* grads) {
  if (!st || (n_req && !energies)) return fail(QF_EINVAL, "NULL argument");
  if (n_req && n_par && !t) return fail(QF_EINVAL, "NULL array");
  if (n_req == 0) return QF_OK;
  trim_plans(st);
  bool done = false;
  size_t r0 = 0;
  qf_status s = multi_small(st, det, ansatz, n_rot, t, n_par, 0, n_req, terms, n_terms, energies, grads, &done);
  if (s != QF_OK || done) return s;
  // not planned yet on this handle (or not the small form): the first request
  // through qf_energy_grad, which validates and plans, then the rest at once
  s = energy_grad_impl(st, det, ansatz, n_rot, t, n_par, terms, n_terms, &energies[0], grads, nullptr, 0, nullptr);
  if (s != QF_OK) return s;
  r0 = 1;
  s = multi_small(st, det, ansatz, n_rot, t, n_par, r0, n_req, terms, n_terms, energies, grads, &done);
  if (s != QF_OK || done) return s;
  for (size_t q = r0; q < n_req; ++q) {
    s = energy_grad_impl(st, det, ansatz, n_rot, t + q * n_par, n_par, terms, n_terms, &energies[q],
                         grads ? grads + q * n_par : nullptr, nullptr, 0, nullptr);
    if (s != QF_OK) return s;
  }
  return QF_OK;
}

qf_status qf_pool_gradients(qf_state* st, uint64_t det, const qf_arot* ansatz, size_t n_rot, const double* t,
                            size_t n_par, const qf_term* terms, size_t n_terms, const qf_arot* pool, size_t n_pool_rot,
                            size_t n_pool, double* energy, double* pool_grad) {
  bool fallback = false;
  qf_status s = energy_grad_impl(st, det, ansatz, n_rot, t, n_par, terms, n_terms, energy, nullptr, nullptr, 0,
                                 nullptr, pool, n_pool_rot, n_pool, pool_grad, &fallback);
  if (s != QF_OK || !fallback) return s;
  // general route: the pool appended to the ansatz at zero angle, whose gradient
  // with respect to the appended parameters is the pool gradient
  if (n_pool && !pool_grad) return fail(QF_EINVAL, "NULL array");
  std::vector<qf_arot> all(ansatz, ansatz + n_rot);
  for (size_t k = 0; k < n_pool_rot; ++k) {
    qf_arot a = pool[k];
    a.param += (int32_t)n_par;
    all.push_back(a);
  }
  std::vector<double> tt(t, t + n_par), g(n_par + n_pool);
  tt.resize(n_par + n_pool, 0.0);
  s = energy_grad_impl(st, det, all.data(), all.size(), tt.data(), n_par + n_pool, terms, n_terms, energy, g.data(),
                       nullptr, 0, nullptr);
  if (s != QF_OK) return s;
  for (size_t k = 0; k < n_pool; ++k) pool_grad[k] = g[n_par + k];
  return QF_OK;
}

qf_status qf_residuals(qf_state* st, uint64_t det, const qf_arot* ansatz, size_t n_rot, const double* t,
                       size_t n_par, const qf_term* terms, size_t n_terms, const uint64_t* dets, size_t n_dets,
                       double* energy, double* grad, double* res) {
  return energy_grad_impl(st, det, ansatz, n_rot, t, n_par, terms, n_terms, energy, grad, dets, n_dets, res);
}

qf_status qf_state_fold_scale(qf_state* st) {
  if (!st) return fail(QF_EINVAL, "state is NULL");
  if (st->scale != 1.0) {
    QF_CUDA(qf::launch_scale(st->psi, st->n, st->dt, st->scale, st->stream));
    st->scale = 1.0;
  }
  return QF_OK;
}

qf_status qf_state_copy_to_host(qf_state* st, void* host, size_t bytes) {
  if (!st || !host) return fail(QF_EINVAL, "NULL argument");
  if (bytes != st->bytes()) return fail(QF_EINVAL, "byte count does not match the state");
  qf_status f = qf_state_fold_scale(st);
  if (f != QF_OK) return f;
  QF_CUDA(d2h(host, st->psi, bytes, st->stream));
  QF_CUDA(cudaStreamSynchronize(st->stream));
  return QF_OK;
}

qf_status qf_state_copy_from_host(qf_state* st, const void* host, size_t bytes) {
  if (!st || !host) return fail(QF_EINVAL, "NULL argument");
  if (bytes != st->bytes()) return fail(QF_EINVAL, "byte count does not match the state");
  QF_CUDA(h2d(st->psi, host, bytes, st->stream));
  st->scale = 1.0;
  st->real = false;
  st->sec_a = st->sec_b = -1;
  return QF_OK;
}

qf_status qf_state_set_hpsi_mode(qf_state* st, int mode) {
  if (!st) return fail(QF_EINVAL, "state is NULL");
  if (mode != QF_HPSI_FP64 && mode != QF_HPSI_DS) return fail(QF_EINVAL, "unknown H|psi> mode");
  st->hpsi_mode = mode;
  return QF_OK;
}

qf_status qf_state_clear_plans(qf_state* st) {
  if (!st) return fail(QF_EINVAL, "state is NULL");
  cudaStreamSynchronize(st->stream);
  for (auto& kv : st->plans) free_plan(kv.second);
  st->plans.clear();
  st->ansatz_plans.clear();
  st->parts_key = st->pool_key = st->map_key = 0;  // descriptors on the device belong to no plan now
  return QF_OK;
}

qf_status qf_sweep_run_items(const qf_state* st, uint64_t* items, size_t cap, size_t* n_runs) {
  if (!st || !n_runs) return fail(QF_EINVAL, "NULL argument");
  if (cap && !items) return fail(QF_EINVAL, "items is NULL with cap > 0");
  if (st->run_items.empty()) return fail(QF_EINVAL, "no part-local sweep has run on this state");
  *n_runs = st->run_items.size();
  for (size_t r = 0; r < std::min(cap, st->run_items.size()); ++r) items[r] = st->run_items[r];
  return QF_OK;
}

qf_status qf_selftest_bounded_wait(void* stream, double limit_s) {
  if (!(limit_s > 0.0) || limit_s > 10.0) return fail(QF_EINVAL, "limit_s must be in (0, 10]");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  unsigned* w = nullptr;
  if (cudaMalloc(&w, 4 * sizeof(unsigned)) != cudaSuccess) {
    cudaGetLastError();
    return fail(QF_ENOMEM, "cudaMalloc(self-test words) failed");
  }
  unsigned h[3] = {0, 0, 0};
  cudaError_t e = cudaMemsetAsync(w, 0, 4 * sizeof(unsigned), s);
  if (e == cudaSuccess) e = qf::launch_wait_selftest(w, limit_s, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h, w, sizeof(h), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(w);
  if (e != cudaSuccess) return fail(QF_ECUDA, std::string("bounded-wait self-test: ") + cudaGetErrorString(e));
  if (h[2]) return fail(QF_ETIMEOUT, "bounded wait gave up after its limit (expected)");
  return fail(QF_ECUDA, "bounded wait returned without a timeout");
}

void qf_transfer_bytes(int reset, uint64_t* h2d_bytes, uint64_t* d2h_bytes) {
  if (h2d_bytes) *h2d_bytes = t_h2d;
  if (d2h_bytes) *d2h_bytes = t_d2h;
  if (reset) t_h2d = t_d2h = 0;
}

qf_status qf_profile_begin(unsigned kind_mask) {
  qf::profile_begin(kind_mask);
  return QF_OK;
}

qf_status qf_profile_read(unsigned kind_mask, uint64_t* launches, double* total_ms) {
  QF_CUDA(qf::profile_read(kind_mask, launches, total_ms));
  return QF_OK;
}

qf_status qf_profile_end(void) {
  qf::profile_end();
  return QF_OK;
}

qf_status qf_state_info(const qf_state* st, int* n, qf_dtype* dtype, void** dev_ptr, double* scale) {
  if (!st) return fail(QF_EINVAL, "state is NULL");
  if (n) *n = st->n;
  if (dtype) *dtype = st->dt;
  if (dev_ptr) *dev_ptr = st->psi;
  if (scale) *scale = st->scale;
  return QF_OK;
}

}  // extern "C"
