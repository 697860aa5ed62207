// Sector-restricted kernels.
//
// A state built from a basis determinant by particle-number- and S_z-
// conserving blocks (every spin-conserving dUCC excitation, Eq. 19) has nonzero
// amplitudes only on determinants with the reference's number of occupied even
// qubits (alpha spin orbitals) and odd qubits (beta): C(n/2, N_a) * C(n/2, N_b)
// of the 2^n basis states, 5 % at 24 qubits.  Restricting the state to that
// sector is the speed-up the paper's conclusion proposes for larger systems.
// Two layouts: in the state's own full 2^n layout these kernels enumerate the
// sector members by combinatorial unranking and never touch the (exactly zero)
// amplitudes outside it; in the compact layout (SecCompact) the members are
// stored contiguously by rank, which keeps a 24-qubit sector (0.85 M members,
// 13.7 MB complex) resident in L2 where the full layout scatters it over
// 0.85 M separate cache lines.
//
// * k_sector_sweep: every excitation block of a circuit in one persistent
//   cooperative launch over the full layout, with a grid barrier between
//   consecutive blocks (qf_apply_circuit).
// * k_sector_run: the part-local sweeps of an energy and gradient evaluation
//   (compact layout, forward and reverse with the gradient overlaps).
// * k_sector_hpsi: lambda = H psi on the sector members only (the only part
//   that enters <psi|lambda>, the gradient overlaps and the reverse sweep, since
//   psi and every block stay in the sector), with <psi|lambda> and <psi|psi>.
//
// Grid barriers spin with an iteration limit; on timeout a block raises the
// error flag and every block leaves at its next barrier.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <mutex>

#include "qf_internal.h"

namespace qf {
namespace {

constexpr int kBinom = 18;  // C(m, k) for m, k < 18 (up to 34 qubits: 17 per parity)

__device__ __forceinline__ unsigned par64s(uint64_t v) { return (unsigned)__popcll(v) & 1u; }

// Binomial tables, built at compile time: c[m][k] = C(m, k) (Pascal's rule; 0
// for k > m) and cs[m][k] = sum of C(m, k') over k' < k, where the size-k group
// of the subsets of m positions starts in a strings table ordered by size.
struct BinomTables {
  uint32_t c[kBinom][kBinom];
  uint32_t cs[kBinom][kBinom];
};
constexpr BinomTables make_binom_tables() {
  BinomTables t{};
  for (int m = 0; m < kBinom; ++m)
    for (int k = 0; k < kBinom; ++k)
      t.c[m][k] = k == 0 ? 1u : (m == 0 ? 0u : t.c[m - 1][k - 1] + t.c[m - 1][k]);
  for (int m = 0; m < kBinom; ++m) {
    uint32_t s = 0;
    for (int k = 0; k < kBinom; ++k) {
      t.cs[m][k] = s;
      s += t.c[m][k];
    }
  }
  return t;
}
constexpr BinomTables kBinomTables = make_binom_tables();
static_assert(kBinomTables.c[17][8] == 24310u && kBinomTables.c[5][7] == 0u && kBinomTables.cs[4][2] == 5u,
              "binomial tables");
__constant__ BinomTables c_binom = kBinomTables;

// Copies of the tables in shared memory (per-thread indices differ, which
// constant memory would serialise).
__device__ void fill_binom(uint32_t (*C)[kBinom]) {
  for (int i = threadIdx.x; i < kBinom * kBinom; i += blockDim.x) (&C[0][0])[i] = (&c_binom.c[0][0])[i];
}

// The r-th k-subset (colex order) of the m positions pos[0..m), as a bit mask.
__device__ __forceinline__ uint64_t unrank(uint32_t r, const uint8_t* pos, int m, int k,
                                           const uint32_t (*C)[kBinom]) {
  uint64_t bits = 0;
  for (int j = m - 1; j >= 0 && k > 0; --j) {
    const uint32_t c = C[j][k];
    if (r >= c) {
      bits |= 1ull << pos[j];
      r -= c;
      --k;
    }
  }
  return bits;
}

__device__ __forceinline__ unsigned par32s(uint32_t v) { return (unsigned)__popc(v) & 1u; }

// Compact index of the member with local alpha / beta strings la, lb.
__device__ __forceinline__ uint64_t compact_index(const SecCompact& cm, uint32_t la, uint32_t lb) {
  return (uint64_t)__ldg(cm.ra + la) * cm.cnt_o + __ldg(cm.rb + lb);
}

constexpr int kSweepThreads = 1024;
constexpr uint64_t kBarrierLimitNs = 2000000000ull;  // a grid barrier gives up after 2 s

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Waits (one thread) until *gen differs from `old`, *err is raised, or limit_ns
// passes; on timeout raises *err.  Returns true when the generation changed.
__device__ bool bounded_wait(volatile unsigned* gen, unsigned old, unsigned* err, uint64_t limit_ns) {
  volatile unsigned* verr = err;
  const uint64_t t0 = global_ns();
  while (*gen == old) {
    if (*verr != 0u) return false;
    if (global_ns() - t0 > limit_ns) {
      atomicExch(err, 1u);
      return false;
    }
  }
  return true;
}

// Grid-wide barrier with a bounded wait.  bar[0] counts arrivals and is never
// reset within a launch: the k-th barrier of a grid of G CTAs is passed once it
// reaches k * G, so each CTA pays one fire-and-forget increment and one polling
// loop.  bar[2] is the error flag.  Returns false when the grid must stop.
__device__ bool grid_barrier(unsigned* bar, unsigned target) {
  __shared__ int stop;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();  // release this CTA's writes (ordered after the CTA barrier)
    atomicAdd(bar, 1u);
    volatile unsigned* vcount = bar;
    volatile unsigned* verr = bar + 2;
    const uint64_t t0 = global_ns();
    int st = 0;
    while (*vcount < target) {
      if (*verr != 0u) {
        st = 1;
        break;
      }
      if (global_ns() - t0 > kBarrierLimitNs) {
        atomicExch(bar + 2, 1u);
        st = 1;
        break;
      }
    }
    __threadfence();  // acquire the other CTAs' writes
    stop = st;
  }
  __syncthreads();
  return !stop;
}

// Self-test of the bounded wait: waits on a generation word that nothing
// changes; words[2] must come back raised.
__global__ void k_wait_selftest(unsigned* words, uint64_t limit_ns) {
  if (threadIdx.x == 0 && blockIdx.x == 0) bounded_wait(words + 1, words[1], words + 2, limit_ns);
}

template <typename T> struct SCx;
template <> struct SCx<double> { using V = double2; };
template <> struct SCx<float> { using V = float2; };

// One block on every sector member its outside positions allow (forward
// sweep in the full layout): the two active rows take psi <- psi + (M - I) psi
// with M chosen by the sign class.
template <bool REALST, typename T>
__device__ void sector_block(typename SCx<T>::V* psi, const SecBlk& B, const uint32_t (*C)[kBinom]) {
  using V = typename SCx<T>::V;
  const uint64_t items = (uint64_t)B.cnt_e * (uint64_t)B.cnt_o;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  T* pr = reinterpret_cast<T*>(psi);
  for (uint64_t it = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; it < items; it += stride) {
    const uint32_t i32 = (uint32_t)it;  // items < 2^32 (at most C(17,8)^2)
    const uint32_t ie = i32 / B.cnt_o, io = i32 - ie * B.cnt_o;
    const uint64_t base = unrank(ie, B.epos, B.ne, B.ke, C) | unrank(io, B.opos, B.no, B.ko, C);
    unsigned cls = 0;
    if (B.nzc > 0) cls = par64s(B.zc[0] & base);
    if (B.nzc > 1) cls |= par64s(B.zc[1] & base) << 1;
    const uint64_t i0 = base | B.pat[0], i1 = base | B.pat[1];
    const T a00 = (T)B.m[cls][0][0], a01 = (T)B.m[cls][0][1], a10 = (T)B.m[cls][1][0], a11 = (T)B.m[cls][1][1];
    // L2-coherent accesses: other SMs wrote these amplitudes before the last grid barrier
    if (REALST) {
      const T v0 = __ldcg(pr + 2 * i0), v1 = __ldcg(pr + 2 * i1);
      __stcg(pr + 2 * i0, fma(a00, v0, fma(a01, v1, v0)));
      __stcg(pr + 2 * i1, fma(a10, v0, fma(a11, v1, v1)));
    } else {
      const V v0 = __ldcg(psi + i0), v1 = __ldcg(psi + i1);
      V o0, o1;
      o0.x = fma(a00, v0.x, fma(a01, v1.x, v0.x));
      o0.y = fma(a00, v0.y, fma(a01, v1.y, v0.y));
      o1.x = fma(a10, v0.x, fma(a11, v1.x, v1.x));
      o1.y = fma(a10, v0.y, fma(a11, v1.y, v1.y));
      __stcg(psi + i0, o0);
      __stcg(psi + i1, o1);
    }
  }
}

__device__ double block_sum_s(double v) {
  __shared__ double red[32];
  __syncthreads();
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) red[wid] = v;
  __syncthreads();
  const int nw = (blockDim.x + 31) >> 5;
  v = (threadIdx.x < nw) ? red[threadIdx.x] : 0.0;
  if (wid == 0) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  }
  return v;
}

// Persistent forward sweep over blocks [0, nblk) in the full layout.  The next
// block's descriptor is loaded while the current one runs.  A one-CTA grid
// needs no grid barrier.
constexpr int kDescWords = sizeof(SecBlk) / 4;
static_assert(sizeof(SecBlk) % 4 == 0 && kDescWords <= 1024, "descriptor copy layout");

template <bool REALST, typename T>
__global__ void __launch_bounds__(kSweepThreads) k_sector_sweep(typename SCx<T>::V* psi,
                                                                const SecBlk* __restrict__ blks, int nblk,
                                                                unsigned* bar) {
  __shared__ uint32_t C[kBinom][kBinom];
  __shared__ SecBlk sb[2];  // current and next block descriptions
  fill_binom(C);
  const int tid = threadIdx.x;
  if (tid < kDescWords) reinterpret_cast<uint32_t*>(&sb[0])[tid] = __ldcg(reinterpret_cast<const uint32_t*>(blks) + tid);
  __syncthreads();
  for (int s = 0; s < nblk; ++s) {
    uint32_t nxt = 0;
    if (s + 1 < nblk && tid < kDescWords) nxt = __ldcg(reinterpret_cast<const uint32_t*>(blks + s + 1) + tid);
    sector_block<REALST, T>(psi, sb[s & 1], C);
    if (s + 1 < nblk) {
      if (tid < kDescWords) reinterpret_cast<uint32_t*>(&sb[(s + 1) & 1])[tid] = nxt;
      if (gridDim.x == 1) {
        __syncthreads();
      } else if (!grid_barrier(bar, (unsigned)(s + 1) * gridDim.x)) {
        return;
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Part-local sweeps (RunInfo / RunPart / RunBlk): one launch per run, one CTA
// per part.  The CTA gathers its part's members from the compact state into
// shared memory, applies every block of the run there (a CTA barrier between
// blocks), and scatters them back.

// The r-th k-subset (colex order) of positions pos[0..m), as a mask of the
// position values.
__device__ __forceinline__ uint32_t unrank_m(uint32_t r, const uint8_t* pos, int m, int k,
                                            const uint32_t (*C)[kBinom]) {
  uint32_t bits = 0;
  for (int j = m - 1; j >= 0 && k > 0; --j) {
    const uint32_t c = C[j][k];
    if (r >= c) {
      bits |= 1u << pos[j];
      r -= c;
      --k;
    }
  }
  return bits;
}

// Sums of FP64 values on the integer pipes (GB300 runs FP64 at 1/64 of FP32, and
// a reduction tree is a serial chain of FP64 adds).  A double is its 53-bit
// integer significand times 2^(e - 1075), e its biased exponent.  Lanes align
// their significands on the warp's largest e, dropping bits below 2^-52 of the
// largest value, and the aligned integers are added exactly in three 21-bit
// slices by single-instruction warp reductions.

// Exact warp sum of m (|m| < 2^58 on every lane).
__device__ __forceinline__ long long warp_add_i64(long long m) {
  const unsigned lo = (unsigned)(m & 0x1FFFFFll), mid = (unsigned)((m >> 21) & 0x1FFFFFll);
  const int hi = (int)(m >> 42);
  const unsigned slo = __reduce_add_sync(0xffffffffu, lo);
  const unsigned smid = __reduce_add_sync(0xffffffffu, mid);
  const int shi = __reduce_add_sync(0xffffffffu, hi);
  return (long long)shi * (1ll << 42) + (long long)smid * (1ll << 21) + (long long)slo;
}

// The warp's sum of v as t * 2^(*e - 1075), |t| < 2^58 (zero and subnormal lanes
// add nothing; the error is at most 32 units of 2^(*e - 1075)).
__device__ __forceinline__ long long warp_sum_fixed(double v, int* e) {
  const long long b = __double_as_longlong(v);
  const int ex = (int)((b >> 52) & 0x7FF);
  const int emax = (int)__reduce_max_sync(0xffffffffu, (unsigned)ex);
  long long m = (ex == 0) ? 0ll : ((b & 0xFFFFFFFFFFFFFll) | 0x10000000000000ll);
  const int sh = emax - ex;
  m = sh > 62 ? 0ll : (m >> sh);
  if (b < 0) m = -m;
  *e = emax;
  return warp_add_i64(m);
}

// The same for a double-single value hi + lo held as two floats: a float is its
// 24-bit significand times 2^(e - 150); both parts are aligned, with 29 guard
// bits, on the warp's largest hi exponent (lo keeps its leading bits down to
// 2^-53 of the largest value) and added exactly.  The sum is t * 2^(*e - 179),
// |t| < 2^59, so the sums of up to twelve warps (a run CTA has at most 384
// threads) stay below 1.5 * 2^62.
__device__ __forceinline__ long long f_aligned(float v, int emax) {
  const int b = __float_as_int(v);
  const int ex = (b >> 23) & 0xFF;
  if (ex == 0) return 0ll;  // zero or subnormal
  const long long m = (long long)((b & 0x7FFFFF) | 0x800000) << 29;
  const int sh = emax - ex;
  const long long a = sh > 62 ? 0ll : (m >> sh);
  return b < 0 ? -a : a;
}
__device__ __forceinline__ long long warp_sum_fixed_ds(float2 v, int* e) {
  const int emax = (int)__reduce_max_sync(0xffffffffu, (unsigned)((__float_as_int(v.x) >> 23) & 0xFF));
  *e = emax - 179 + 1075;  // on the double scale of warp_fixed_to_double: t * 2^(*e - 1075)
  return warp_add_i64(f_aligned(v.x, emax) + f_aligned(v.y, emax));
}

// d * 2^k for -2044 <= k <= 1023, exact unless the result is subnormal.
__device__ __forceinline__ double scale_pow2(double d, int k) {
  if (k < -1022) {
    d *= __longlong_as_double(1ll << 52);  // 2^-1022
    k += 1022;
  }
  return d * __longlong_as_double((long long)(k + 1023) << 52);
}

// Sum of the lanes' (t, e) pairs from warp_sum_fixed (one lane per warp of the CTA nonzero, at most 12) as
// one double: aligned on the largest e, added exactly, converted once.
__device__ __forceinline__ double warp_fixed_to_double(long long t, int e) {
  const int emax = (int)__reduce_max_sync(0xffffffffu, (unsigned)(t != 0 ? e : 0));
  const int sh = emax - e;
  const long long m = (t == 0 || sh > 62) ? 0ll : (t >> sh);
  const long long tot = warp_add_i64(m);
  return tot == 0 ? 0.0 : scale_pow2((double)tot, emax - 1075);
}

// Double-single arithmetic of the part-local sweeps (complex128 in QF_HPSI_DS
// mode): a value is a float pair hi + lo with |lo| <= ulp(hi) / 2, about 48
// significant bits.  Every rounding step is explicit, so that no multiply is
// fused into an error-free transformation.
__device__ __forceinline__ float2 ds_renorm(float s, float e) {  // Fast2Sum (|s| >= |e| or s == 0)
  const float h = __fadd_rn(s, e);
  return make_float2(h, __fsub_rn(e, __fsub_rn(h, s)));
}
// a * b as an unnormalised pair: the rounded product of the high parts and, in
// the low part, its exact error plus both cross terms.
__device__ __forceinline__ float2 ds_prod(float2 a, float2 b) {
  const float ph = __fmul_rn(a.x, b.x);
  float pl = fmaf(a.x, b.x, -ph);
  pl = fmaf(a.x, b.y, pl);
  pl = fmaf(a.y, b.x, pl);
  return make_float2(ph, pl);
}
// TwoSum: s + *e == a + b exactly.
__device__ __forceinline__ float two_sum(float a, float b, float* e) {
  const float s = __fadd_rn(a, b);
  const float bp = __fsub_rn(s, a);
  *e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bp)), __fsub_rn(b, bp));
  return s;
}
// x + p + q for p, q from ds_prod: the high parts through two TwoSums, the low
// parts and both errors summed in float, one renormalisation (27 operations per
// output; normalising each product and partial sum would take 36).
__device__ __forceinline__ float2 ds_sum3(float2 x, float2 p, float2 q) {
  float e1, e2;
  const float s1 = two_sum(x.x, p.x, &e1);
  const float s2 = two_sum(s1, q.x, &e2);
  return ds_renorm(s2, __fadd_rn(__fadd_rn(__fadd_rn(x.y, p.y), __fadd_rn(q.y, e1)), e2));
}
// c + a x + b y (one output of a 2x2 block rotation, m = composite - identity)
__device__ __forceinline__ float2 ds_rot(float2 a, float2 x, float2 b, float2 y, float2 c) {
  return ds_sum3(c, ds_prod(a, x), ds_prod(b, y));
}
// p + q for p, q from ds_prod (or normalised pairs), renormalised.
__device__ __forceinline__ float2 ds_sum2(float2 p, float2 q) {
  float e;
  const float s = two_sum(p.x, q.x, &e);
  return ds_renorm(s, __fadd_rn(e, __fadd_rn(p.y, q.y)));
}
__device__ __forceinline__ float2 ds_of(double v) {
  const float hi = __double2float_rn(v);
  return make_float2(hi, __double2float_rn(v - (double)hi));
}

constexpr int kRunThreads = 256;  // threads of a part-local run CTA (item maps, FP64 and FP32 sweeps)
constexpr int kRunBlkWords = sizeof(RunBlk) / 4;
// Threads of a mapped sweep CTA (forward, and logged reverse).  A run's time is
// that of its largest parts, whose block steps take ceil(items / threads) item
// rounds each, so these take as many threads as still leave every part of a run
// resident at once (512 parts on 152 SMs: 4 CTAs per SM): 384 for the forward
// (40 registers), 288 for the reverse (56 registers).
template <int MODE>
__host__ __device__ constexpr int wide_threads() {
  return MODE == 0 ? 384 : 288;
}
// Coefficient words a mapped sweep step copies: m then q (FP64) or mf then qf (FP32).
constexpr int kCoefWordsMax = 64;
static_assert(offsetof(RunBlk, q) == offsetof(RunBlk, m) + sizeof(double) * 16 &&
                  offsetof(RunBlk, qf) == offsetof(RunBlk, mf) + sizeof(float) * 16 && kSparseMaxCls == 4 &&
                  offsetof(RunBlk, m) % 8 == 0,
              "coefficient layout of RunBlk");
static_assert(sizeof(RunBlk) % 4 == 0 && kRunBlkWords <= kRunThreads && kRunBlkWords <= 288,
              "run descriptor copy layout");

// Shared-memory bytes per member: psi real parts (forward), (psi, lam) packed
// real pairs (reverse, real), psi and lam complex (reverse, complex), or lam's
// real parts (reverse, real, psi read from the forward log); plus the member's
// compact index, kept for the scatter (the read-only MODE 4 has none).
template <int MODE, typename T>
__host__ __device__ constexpr size_t run_member_bytes() {
  return (MODE == 0 || MODE == 3 ? sizeof(T) : (MODE == 1 || MODE == 4) ? 2 * sizeof(T) : 4 * sizeof(T)) +
         (MODE == 4 ? 0 : sizeof(uint32_t));
}
__host__ __device__ inline size_t align16(size_t b) { return (b + 15) & ~(size_t)15; }

__device__ void fill_binom_prefix(uint32_t (*Cs)[kBinom]) {
  for (int i = threadIdx.x; i < kBinom * kBinom; i += blockDim.x) (&Cs[0][0])[i] = (&c_binom.cs[0][0])[i];
}

// MODE 0: forward, psi real; with a log, each item's rotated pair (psi_i0,
// psi_i1) is also written to log[P.logbase + offset of the block + item].
// MODE 1: reverse, psi and lam real, packed as (psi, lam) in one complex slot;
// psi is un-rotated block by block.
// MODE 2: reverse, psi and lam complex.
// MODE 3: reverse, lam real (psi's imaginary slots); psi after each block is
// read back from the forward log instead of being un-rotated.
// MODE 4: overlaps only, psi and lam real and packed: every block's overlap on
// the same (psi, lam), nothing rotated or written back (operator-pool gradients).
// Overlaps accumulate in the state's precision (FP64 for complex128, FP32 for
// complex64); each part's overlap with a block is written to partial in FP64.
// Programmatic dependent launch: a sweep launch may start while the previous
// kernel of the stream finishes; it reads only plan data (descriptors, parts,
// coefficients) before grid_dep_wait, which returns once that kernel has
// completed and its writes are visible.  A kernel lets the next launch start
// only after its own wait (so it never overlaps one two places before it).  Both
// are no-ops for a kernel launched without the attribute.
__device__ __forceinline__ void grid_dep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void grid_dep_launch_dependents() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

template <int MODE, typename T, bool DSW, int NT>
__device__ __forceinline__ void sector_run_body(typename SCx<T>::V* psi, typename SCx<T>::V* lam, RunInfo run,
                                                const RunPart* __restrict__ parts, const RunBlk* __restrict__ blks,
                                                double* partial, int pmax, SecCompact cm, typename SCx<T>::V* log,
                                                const uint16_t* __restrict__ strs,
                                                const uint32_t* __restrict__ map, bool dss) {
  using V = typename SCx<T>::V;
  constexpr int NW = NT / 32;
  static_assert(NT % 32 == 0 && NT >= kRunBlkWords && NT <= 384, "run CTA size");
  constexpr bool ADJ = MODE != 0;
  constexpr bool F32 = sizeof(T) == 4;
  extern __shared__ __align__(16) unsigned char dsm[];
  __shared__ uint32_t C[kBinom][kBinom];
  __shared__ uint32_t Cs[kBinom][kBinom];
  __shared__ RunBlk sb[2];
  __shared__ RunInfo R;
  __shared__ RunPart P;
  // every thread's overlap with the last two blocks: block s's values are summed
  // by one warp during block s + 1 and rewritten after block s + 1's barrier
  __shared__ T red[ADJ ? 2 : 1][(ADJ && !DSW) ? NT : 1];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  fill_binom(C);
  fill_binom_prefix(Cs);
  if (tid == 0) {
    R = run;
    P = parts[run.part0 + blockIdx.x];
  }
  const int nb = run.b1 - run.b0;
  auto blk_of = [&](int s) { return ADJ ? run.b1 - 1 - s : run.b0 + s; };
  if (tid < kRunBlkWords)
    reinterpret_cast<uint32_t*>(&sb[0])[tid] = __ldg(reinterpret_cast<const uint32_t*>(blks + blk_of(0)) + tid);
  __syncthreads();
  // shared memory: amplitudes, then compact indices
  const uint32_t cap = R.maxsize;
  T* ar = reinterpret_cast<T*>(dsm);   // MODE 0 (psi), MODE 3 (lam)
  float2* ad = reinterpret_cast<float2*>(dsm);  // the same, double-single (DSW)
  V* av = reinterpret_cast<V*>(dsm);   // MODE 1, 2, 4 (psi)
  V* lv = av + cap;                    // MODE 2 (lam)
  constexpr size_t idx_bytes = MODE == 4 ? 0 : sizeof(uint32_t);
  const size_t amp_bytes = align16((run_member_bytes<MODE, T>() - idx_bytes) * cap);
  uint32_t* gi = reinterpret_cast<uint32_t*>(dsm + amp_bytes);
  const uint32_t size = P.cnta * P.cntb;
  // item-map words of this part's class (forward and logged reverse sweeps)
  const uint32_t* mp = (MODE == 0 || MODE == 3) && map ? map + P.mapbase : nullptr;
  // Mapped sweep tables (plan data only): every step's item count, offset and G
  // class bits, and the first two steps' coefficients.
  __shared__ uint32_t stn[kRunMaxBlocks], sto[kRunMaxBlocks];
  __shared__ uint8_t stc[kRunMaxBlocks];
  __shared__ __align__(16) uint32_t cw[3][kCoefWordsMax];
  constexpr int kCw = DSW ? (MODE == 3 ? 40 : 32) : F32 ? (MODE == 3 ? 20 : 16) : (MODE == 3 ? 64 : 32);
  constexpr size_t kCoff = DSW ? offsetof(RunBlk, md) : F32 ? offsetof(RunBlk, mf) : offsetof(RunBlk, m);
  auto coef_word = [&](int st) {
    return __ldg(reinterpret_cast<const uint32_t*>(reinterpret_cast<const char*>(blks + blk_of(st)) + kCoff) + tid);
  };
  if (mp) {
    for (int f = tid; f < nb; f += NT) {  // f: the block's position in forward order
      const RunBlk* Bg = blks + run.b0 + f;
      const int ne = __ldg(&Bg->ne), no = __ldg(&Bg->no), nzc = __ldg(&Bg->nzc);
      const int ke = P.ka - __ldg(&Bg->e0), ko = P.kb - __ldg(&Bg->o0);
      stn[f] = (ke >= 0 && ke <= ne && ko >= 0 && ko <= no) ? C[ne][ke] * C[no][ko] : 0u;
      unsigned cg = 0;
      if (nzc > 0) cg = par32s(__ldg(&Bg->zg[0][0]) & P.ga) ^ par32s(__ldg(&Bg->zg[0][1]) & P.gb);
      if (nzc > 1) cg |= (par32s(__ldg(&Bg->zg[1][0]) & P.ga) ^ par32s(__ldg(&Bg->zg[1][1]) & P.gb)) << 1;
      stc[f] = (uint8_t)cg;
    }
    if (tid < kCw) {
      cw[0][tid] = coef_word(0);
      if (nb > 1) cw[1][tid] = coef_word(1);
    }
    __syncthreads();
    if (tid == 0) {
      uint32_t a = 0;
      for (int f = 0; f < nb; ++f) {
        sto[f] = a;
        a += stn[f];
      }
    }
  }
  // the state (and the maps, the log) come from earlier kernels of the stream
  grid_dep_wait();
  // the real slot each member moves: psi's real part (MODE 0), lam's in psi's imaginary slot (MODE 3)
  const int slot = MODE == 3 ? 1 : 0;
  const T* pr = reinterpret_cast<const T*>(psi);
  for (uint32_t m = tid; m < size; m += NT) {
    const uint32_t ia = m / P.cntb, ib = m - ia * P.cntb;
    const uint32_t sa = unrank_m(ia, R.apos, R.ua, P.ka, C) | P.ga;
    const uint32_t sbm = unrank_m(ib, R.bpos, R.ub, P.kb, C) | P.gb;
    const uint32_t g = (uint32_t)compact_index(cm, sa, sbm);
    if (MODE != 4) gi[m] = g;
    if (DSW) {  // double-single state layout (dss): the slot already holds the (hi, lo) pair
      ad[m] = dss ? __ldcg(reinterpret_cast<const float2*>(psi) + 2 * (size_t)g + slot)
                  : ds_of(__ldcg(pr + 2 * (size_t)g + slot));
    } else if (MODE == 0 || MODE == 3) {
      ar[m] = __ldcg(pr + 2 * (size_t)g + slot);
    } else {
      av[m] = __ldcg(psi + g);
      if (MODE == 2) lv[m] = __ldcg(lam + g);
    }
  }
  // items of a block in this part (uniform over the CTA)
  auto items_of = [&](const RunBlk& B) -> uint64_t {
    const int ke = P.ka - B.e0, ko = P.kb - B.o0;
    if (ke < 0 || ke > B.ne || ko < 0 || ko > B.no) return 0;
    return (uint64_t)C[B.ne][ke] * C[B.no][ko];
  };
  // log offset of the current block within this part's log
  uint64_t logoff = 0;
  if (MODE == 3 && !mp) {  // the reverse starts past the part's last block
    for (int s = 0; s < nb; ++s) {
      const RunBlk* Bg = blks + run.b0 + s;
      const int ne = __ldg(&Bg->ne), no = __ldg(&Bg->no);
      const int ke = P.ka - __ldg(&Bg->e0), ko = P.kb - __ldg(&Bg->o0);
      if (ke >= 0 && ke <= ne && ko >= 0 && ko <= no) logoff += (uint64_t)C[ne][ke] * C[no][ko];
    }
  }
  __syncthreads();
  // The overlap of block ps with this part: the threads' values in red[ps & 1],
  // summed by one warp (rotating over the upper warps, which hold items least
  // often) over the rows of the pw warps that had items, in warp order, then
  // lane order by a butterfly.  Deterministic.
  auto reduce_block = [&](int ps, int pw) {
    if (warp != NW - 1 - (ps & 3)) return;
    T v = T(0);
    if (pw > 0) {
      const T* rr = red[ps & 1];
      v = rr[lane];
      for (int j = 1; j < pw; ++j) v += rr[32 * j + lane];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    }
    if (lane == 0) partial[(size_t)blk_of(ps) * pmax + blockIdx.x] = (double)v;
  };
  int pend_w = 0;  // warps with items in the previous block (its overlaps wait in red)
  // MODE 3: the log pair of item tid of the current block, loaded during the
  // previous block so that its DRAM latency overlaps that block's barrier; the
  // item-map word of item tid likewise (MODE 0 and 3)
  V pre{};
  bool pre_ok = false;
  if (mp) {
    // Mapped sweep (forward, and reverse with the log): each step runs its items
    // from the class's map with its block's coefficients.  Item counts, offsets and
    // G class bits of every step are tabulated first; the coefficients, map words
    // and log pairs of a step are loaded two steps ahead, so no load latency sits
    // between two barriers.  A complex128 reverse sums each step's overlaps on the
    // integer pipes (warp_sum_fixed), one step later, with no FP64 chain.
    __shared__ long long wtot[2][NW];  // per-warp overlap sums of the last two steps
    __shared__ int wexp[2][NW];
    using LV = typename std::conditional<DSW, float4, V>::type;  // a log pair
    constexpr bool IRED = MODE == 3 && !F32;  // integer overlap reduction
    LV* lgp = log ? reinterpret_cast<LV*>(log + P.logbase) : nullptr;
    auto pos = [&](int st) { return MODE == 3 ? nb - 1 - st : st; };  // a step's forward position
    // item tid of step s (wq0, lq0) and of step s + 1 (wq1, lq1): map word and
    // (reverse) log pair
    uint32_t wq0 = 0u, wq1 = 0u;
    LV lq0{}, lq1{};
    if ((uint32_t)tid < stn[pos(0)]) {
      wq0 = __ldg(mp + sto[pos(0)] + tid);
      if (MODE == 3) lq0 = __ldcs(lgp + sto[pos(0)] + tid);
    }
    if (nb > 1 && (uint32_t)tid < stn[pos(1)]) {
      wq1 = __ldg(mp + sto[pos(1)] + tid);
      if (MODE == 3) lq1 = __ldcs(lgp + sto[pos(1)] + tid);
    }
    uint32_t nxtc = 0;  // coefficient word of step s + 2, stored at step s + 1
    if (nb > 2 && tid < kCw) nxtc = coef_word(2);
    // the previous step's per-warp sums, combined by one warp into the block's partial
    auto reduce_fixed = [&](int ps, int pw) {
      if (warp != NW - 1 - (ps & 3)) return;
      const long long t = lane < pw ? wtot[ps & 1][lane] : 0ll;
      const int e = lane < pw ? wexp[ps & 1][lane] : 0;
      const double v = warp_fixed_to_double(t, e);
      if (lane == 0) partial[(size_t)blk_of(ps) * pmax + blockIdx.x] = v;
    };
    for (int s = 0; s < nb; ++s) {
      const int f = pos(s);
      if (s >= 1 && s + 1 < nb && tid < kCw) {  // step s + 1's coefficients, loaded during step s - 1
        cw[(s + 1) % 3][tid] = nxtc;
        nxtc = (s + 2 < nb) ? coef_word(s + 2) : 0u;
      }
      if (ADJ && s > 0) {
        if (IRED) reduce_fixed(s - 1, pend_w);
        else reduce_block(s - 1, pend_w);
      }
      const uint32_t n_s = stn[f], o_s = sto[f];
      const unsigned cg = stc[f];
      const T* cf = reinterpret_cast<const T*>(cw[s % 3]);  // m[cls][i][j] at 4 cls + 2 i + j, then q or qf
      const uint32_t wnow = wq0;
      const LV lnow = lq0;
      T acc = T(0);
      float2 dacc = make_float2(0.0f, 0.0f);  // DSW overlap
      for (uint32_t it = tid; it < n_s; it += NT) {
        const bool first = it == (uint32_t)tid;
        const uint32_t w = first ? wnow : __ldg(mp + o_s + it);
        const uint32_t i0 = w & 0xFFFu, i1 = (w >> 12) & 0xFFFu;
        const unsigned cls = cg ^ (w >> 24);
        if constexpr (DSW) {
          const float2* cd = reinterpret_cast<const float2*>(cw[s % 3]);  // md, then qd
          const float4 da = reinterpret_cast<const float4*>(cd)[2 * cls];      // md[cls][0][0..1]
          const float4 db = reinterpret_cast<const float4*>(cd)[2 * cls + 1];  // md[cls][1][0..1]
          const float2 d00 = make_float2(da.x, da.y), d01 = make_float2(da.z, da.w);
          const float2 d10 = make_float2(db.x, db.y), d11 = make_float2(db.z, db.w);
          const float2 x0 = ad[i0], x1 = ad[i1];
          if (MODE == 3) {
            const float4 pq = first ? lnow : __ldcs(lgp + o_s + it);  // psi pair after this block
            const float2 p0 = make_float2(pq.x, pq.y), p1 = make_float2(pq.z, pq.w);
            // Im <lam|Q|psi> on the pair: q01 (lam0 psi1 - lam1 psi0)
            const float2 t = ds_sum2(ds_prod(x0, p1), ds_prod(make_float2(-x1.x, -x1.y), p0));
            dacc = ds_sum2(dacc, ds_prod(cd[16 + cls], t));
          }
          const float2 o0 = ds_rot(d00, x0, d01, x1, x0), o1 = ds_rot(d10, x0, d11, x1, x1);
          ad[i0] = o0;
          ad[i1] = o1;
          if (MODE == 0 && lgp) __stcs(lgp + o_s + it, make_float4(o0.x, o0.y, o1.x, o1.y));
        } else {
          const T a00 = cf[4 * cls], a01 = cf[4 * cls + 1], a10 = cf[4 * cls + 2], a11 = cf[4 * cls + 3];
          if (MODE == 0) {
            const T v0 = ar[i0], v1 = ar[i1];
            const T o0 = fma(a00, v0, fma(a01, v1, v0)), o1 = fma(a10, v0, fma(a11, v1, v1));
            ar[i0] = o0;
            ar[i1] = o1;
            if (lgp) {
              V wv;
              wv.x = o0;
              wv.y = o1;
              __stcs(lgp + o_s + it, wv);  // streamed: read back once by the reverse sweep
            }
          } else {
            const T q01 = F32 ? cf[16 + cls] : cf[16 + 4 * cls + 1];
            const V pp = first ? lnow : __ldcs(lgp + o_s + it);
            const T w0 = ar[i0], w1 = ar[i1];
            // Im <lam|Q|psi> on the pair, Qi = [[0, q01], [-q01, 0]] (checked on the host)
            acc = fma(q01, fma(w0, pp.y, -w1 * pp.x), acc);
            ar[i0] = fma(a00, w0, fma(a01, w1, w0));
            ar[i1] = fma(a10, w0, fma(a11, w1, w1));
          }
        }  // DSW
      }
      if (ADJ) {
        pend_w = n_s >= (uint32_t)NT ? NW : (int)((n_s + 31) / 32);
        if (IRED) {
          if (warp < pend_w) {  // warps past pend_w hold no items this step
            int e;
            const long long t = DSW ? warp_sum_fixed_ds(dacc, &e) : warp_sum_fixed((double)acc, &e);
            if (lane == 0) {
              wtot[s & 1][warp] = t;
              wexp[s & 1][warp] = e;
            }
          }
        } else {
          red[s & 1][tid] = acc;
        }
      }
      wq0 = wq1;
      lq0 = lq1;
      if (s + 2 < nb) {  // item tid of step s + 2
        const int f2 = pos(s + 2);
        if ((uint32_t)tid < stn[f2]) {
          wq1 = __ldg(mp + sto[f2] + tid);
          if (MODE == 3) lq1 = __ldcs(lgp + sto[f2] + tid);
        }
      }
      __syncthreads();
    }
    if (ADJ && nb > 0) {
      if (IRED) reduce_fixed(nb - 1, pend_w);
      else reduce_block(nb - 1, pend_w);
    }

  } else
  for (int s = 0; s < nb; ++s) {
    uint32_t nxt = 0;
    if (s + 1 < nb && tid < kRunBlkWords)
      nxt = __ldg(reinterpret_cast<const uint32_t*>(blks + blk_of(s + 1)) + tid);
    int ne1 = 0, no1 = 0, e01 = 0, o01 = 0;  // MODE 3: the next block's item geometry
    if (MODE == 3 && s + 1 < nb) {
      const RunBlk* Bn = blks + blk_of(s + 1);
      ne1 = __ldg(&Bn->ne);
      no1 = __ldg(&Bn->no);
      e01 = __ldg(&Bn->e0);
      o01 = __ldg(&Bn->o0);
    }
    if (ADJ && s > 0) reduce_block(s - 1, pend_w);
    const RunBlk& B = sb[s & 1];
    T acc = T(0);
    const int ke = P.ka - B.e0, ko = P.kb - B.o0;
    const uint64_t nitems = items_of(B);
    if (MODE == 3) logoff -= nitems;
    if (nitems) {
      const uint32_t co = C[B.no][ko];
      const uint32_t items = (uint32_t)nitems;
      unsigned cg = 0;  // sign-class bits from the part's occupation of G
      if (B.nzc > 0) cg = par32s(B.zg[0][0] & P.ga) ^ par32s(B.zg[0][1] & P.gb);
      if (B.nzc > 1) cg |= (par32s(B.zg[1][0] & P.ga) ^ par32s(B.zg[1][1] & P.gb)) << 1;
      V* lg = ((MODE == 0 || MODE == 3) && log) ? log + P.logbase + logoff : nullptr;
      // the block's outside strings of sizes ke and ko, when tabulated
      const bool tab = strs && B.lsa != kNoStrings;
      const uint32_t sa0 = tab ? B.lsa + Cs[B.ne][ke] : 0u;
      const uint32_t sb0 = tab ? B.lsb + Cs[B.no][ko] : 0u;
      const float inv_co = __frcp_rn((float)co);  // items < 2^24: the estimate is off by at most one
      for (uint32_t it = tid; it < items; it += NT) {
        uint32_t ie = (uint32_t)((float)it * inv_co);
        if (ie * co > it) --ie;
        else if ((ie + 1) * co <= it) ++ie;
        const uint32_t io = it - ie * co;
        const uint32_t la = tab ? (uint32_t)__ldg(strs + sa0 + ie) : unrank_m(ie, B.epos, B.ne, ke, C);
        const uint32_t lb = tab ? (uint32_t)__ldg(strs + sb0 + io) : unrank_m(io, B.opos, B.no, ko, C);
        unsigned cls = cg;
        if (B.nzc > 0) cls ^= par32s(B.zu[0][0] & la) ^ par32s(B.zu[0][1] & lb);
        if (B.nzc > 1) cls ^= (par32s(B.zu[1][0] & la) ^ par32s(B.zu[1][1] & lb)) << 1;
        // ranks of run-local strings: the general colex rank table
        const uint32_t i0 = (uint32_t)__ldg(cm.ra + (la | B.pu[0][0])) * P.cntb + __ldg(cm.ra + (lb | B.pu[0][1]));
        const uint32_t i1 = (uint32_t)__ldg(cm.ra + (la | B.pu[1][0])) * P.cntb + __ldg(cm.ra + (lb | B.pu[1][1]));
        T a00, a01, a10, a11, q01;
        if constexpr (F32) {
          a00 = B.mf[cls][0][0], a01 = B.mf[cls][0][1], a10 = B.mf[cls][1][0], a11 = B.mf[cls][1][1];
          q01 = B.qf[cls];
        } else {
          a00 = B.m[cls][0][0], a01 = B.m[cls][0][1], a10 = B.m[cls][1][0], a11 = B.m[cls][1][1];
          q01 = B.q[cls][0][1];
        }
        if (MODE == 0) {
          const T v0 = ar[i0], v1 = ar[i1];
          const T o0 = fma(a00, v0, fma(a01, v1, v0)), o1 = fma(a10, v0, fma(a11, v1, v1));
          ar[i0] = o0;
          ar[i1] = o1;
          if (lg) {
            V w;
            w.x = o0;
            w.y = o1;
            __stcs(lg + it, w);  // streamed: read back once by the reverse sweep
          }
        } else if (MODE == 3) {
          // psi on the pair after this block (forward log)
          const V pp = (pre_ok && it == (uint32_t)tid) ? pre : __ldcs(lg + it);
          const T w0 = ar[i0], w1 = ar[i1];
          // Im <lam|Q|psi> on the pair, Qi = [[0, q01], [-q01, 0]] (checked on the host)
          acc = fma(q01, fma(w0, pp.y, -w1 * pp.x), acc);
          ar[i0] = fma(a00, w0, fma(a01, w1, w0));
          ar[i1] = fma(a10, w0, fma(a11, w1, w1));
        } else if (MODE == 4) {
          const V p0 = av[i0], p1 = av[i1];  // (psi, lambda)
          acc = fma(q01, fma(p0.y, p1.x, -p1.y * p0.x), acc);
        } else if (MODE == 1) {
          const V p0 = av[i0], p1 = av[i1];  // (psi, lambda)
          // Im <lam|Q|psi> on the pair, Qi = [[0, q01], [-q01, 0]] (checked on the host)
          acc = fma(q01, fma(p0.y, p1.x, -p1.y * p0.x), acc);
          V o0, o1;
          o0.x = fma(a00, p0.x, fma(a01, p1.x, p0.x));
          o0.y = fma(a00, p0.y, fma(a01, p1.y, p0.y));
          o1.x = fma(a10, p0.x, fma(a11, p1.x, p1.x));
          o1.y = fma(a10, p0.y, fma(a11, p1.y, p1.y));
          av[i0] = o0;
          av[i1] = o1;
        } else {
          const V v0 = av[i0], v1 = av[i1], w0 = lv[i0], w1 = lv[i1];
          const double q00 = B.q[cls][0][0], q10 = B.q[cls][1][0], q11 = B.q[cls][1][1];
          const double qq01 = B.q[cls][0][1];
          double t = (double)w0.x * (q00 * v0.x + qq01 * v1.x) + (double)w0.y * (q00 * v0.y + qq01 * v1.y);
          t += (double)w1.x * (q10 * v0.x + q11 * v1.x) + (double)w1.y * (q10 * v0.y + q11 * v1.y);
          acc += (T)t;
          V o0, o1;
          o0.x = fma(a00, w0.x, fma(a01, w1.x, w0.x));
          o0.y = fma(a00, w0.y, fma(a01, w1.y, w0.y));
          o1.x = fma(a10, w0.x, fma(a11, w1.x, w1.x));
          o1.y = fma(a10, w0.y, fma(a11, w1.y, w1.y));
          lv[i0] = o0;
          lv[i1] = o1;
          o0.x = fma(a00, v0.x, fma(a01, v1.x, v0.x));
          o0.y = fma(a00, v0.y, fma(a01, v1.y, v0.y));
          o1.x = fma(a10, v0.x, fma(a11, v1.x, v1.x));
          o1.y = fma(a10, v0.y, fma(a11, v1.y, v1.y));
          av[i0] = o0;
          av[i1] = o1;
        }
      }
    }
    if (MODE == 0) logoff += nitems;
    if (MODE == 3) {  // the next block's log starts its item count before this one's
      pre_ok = false;
      const int ke1 = P.ka - e01, ko1 = P.kb - o01;
      if (log && s + 1 < nb && ke1 >= 0 && ke1 <= ne1 && ko1 >= 0 && ko1 <= no1) {
        const uint64_t n1 = (uint64_t)C[ne1][ke1] * C[no1][ko1];
        if ((uint64_t)tid < n1) {
          pre = __ldcs(log + P.logbase + (logoff - n1) + tid);
          pre_ok = true;
        }
      }
    }
    if (ADJ) {
      red[s & 1][tid] = acc;
      pend_w = nitems >= (uint64_t)NT ? NW : (int)((nitems + 31) / 32);
    }
    if (s + 1 < nb && tid < kRunBlkWords) reinterpret_cast<uint32_t*>(&sb[(s + 1) & 1])[tid] = nxt;
    __syncthreads();
  }
  if (ADJ && nb > 0 && !mp) reduce_block(nb - 1, pend_w);
  // the next run may launch once every CTA is here (its CTAs then take the SMs as
  // this run's scatters finish, so that they spread over the SMs)
  grid_dep_launch_dependents();
  if (MODE == 4) return;  // read only
  T* pw = reinterpret_cast<T*>(psi);
  for (uint32_t m = tid; m < size; m += NT) {
    const uint32_t g = gi[m];
    if (DSW) {
      const float2 d = ad[m];
      if (dss)
        __stcg(reinterpret_cast<float2*>(psi) + 2 * (size_t)g + slot, d);
      else
        __stcg(pw + 2 * (size_t)g + slot, (T)((double)d.x + (double)d.y));
    } else if (MODE == 0 || MODE == 3) {
      __stcg(pw + 2 * (size_t)g + slot, ar[m]);
    } else {
      __stcg(psi + g, av[m]);
      if (MODE == 2) __stcg(lam + g, lv[m]);
    }
  }
}

// The sweeps: kRunThreads threads, or wide_threads for the mapped forward and
// logged reverse (every double-single sweep is one).
#define QF_RUN_ARGS                                                                                              \
  typename SCx<T>::V *psi, typename SCx<T>::V *lam, RunInfo run, const RunPart *__restrict__ parts,               \
      const RunBlk *__restrict__ blks, double *partial, int pmax, SecCompact cm, typename SCx<T>::V *log,         \
      const uint16_t *__restrict__ strs, const uint32_t *__restrict__ map, bool dss
template <int MODE, typename T>
__global__ void __launch_bounds__(kRunThreads) k_sector_run(QF_RUN_ARGS) {
  sector_run_body<MODE, T, false, kRunThreads>(psi, lam, run, parts, blks, partial, pmax, cm, log, strs, map, dss);
}
template <int MODE, typename T, bool DSW>
__global__ void __launch_bounds__(wide_threads<MODE>()) k_sector_run_wide(QF_RUN_ARGS) {
  sector_run_body<MODE, T, DSW, wide_threads<MODE>()>(psi, lam, run, parts, blks, partial, pmax, cm, log, strs, map,
                                                       dss);
}
#undef QF_RUN_ARGS

// Item maps (RunPart::mapbase): for the part representing each class, every
// forward block's items in sweep order, one word each -- the item's two
// members inside the part and the sign-class bits of its U strings -- computed
// as the sweep itself would (outside strings, colex ranks, class masks).
__global__ void __launch_bounds__(kRunThreads) k_run_itemmap(RunInfo run, const RunPart* __restrict__ parts,
                                                             const RunBlk* __restrict__ blks, SecCompact cm,
                                                             const uint16_t* __restrict__ strs, uint32_t* map) {
  __shared__ uint32_t C[kBinom][kBinom];
  __shared__ uint32_t Cs[kBinom][kBinom];
  fill_binom(C);
  fill_binom_prefix(Cs);
  __syncthreads();
  const RunPart P = parts[run.part0 + blockIdx.x];
  if (!P.maprep) return;
  uint64_t off = 0;
  for (int b = run.b0; b < run.b1; ++b) {
    const RunBlk& B = blks[b];
    const int ke = P.ka - B.e0, ko = P.kb - B.o0;
    if (ke < 0 || ke > B.ne || ko < 0 || ko > B.no) continue;
    const uint32_t co = C[B.no][ko];
    const uint32_t items = C[B.ne][ke] * co;
    const bool tab = strs && B.lsa != kNoStrings;
    const uint32_t sa0 = tab ? B.lsa + Cs[B.ne][ke] : 0u;
    const uint32_t sb0 = tab ? B.lsb + Cs[B.no][ko] : 0u;
    for (uint32_t it = threadIdx.x; it < items; it += blockDim.x) {
      const uint32_t ie = it / co, io = it - ie * co;
      const uint32_t la = tab ? (uint32_t)__ldg(strs + sa0 + ie) : unrank_m(ie, B.epos, B.ne, ke, C);
      const uint32_t lb = tab ? (uint32_t)__ldg(strs + sb0 + io) : unrank_m(io, B.opos, B.no, ko, C);
      unsigned cls = 0;
      if (B.nzc > 0) cls ^= par32s(B.zu[0][0] & la) ^ par32s(B.zu[0][1] & lb);
      if (B.nzc > 1) cls ^= (par32s(B.zu[1][0] & la) ^ par32s(B.zu[1][1] & lb)) << 1;
      const uint32_t i0 = (uint32_t)__ldg(cm.ra + (la | B.pu[0][0])) * P.cntb + __ldg(cm.ra + (lb | B.pu[0][1]));
      const uint32_t i1 = (uint32_t)__ldg(cm.ra + (la | B.pu[1][0])) * P.cntb + __ldg(cm.ra + (lb | B.pu[1][1]));
      map[P.mapbase + off + it] = i0 | (i1 << 12) | (cls << 24);
    }
    off += items;
  }
}

// out[b] = sum over the parts of block b's run of partial[b * pmax + part], in part order.
// One warp per block: lane l sums parts l, l + 32, ... in order, then a fixed
// butterfly combines the lanes (deterministic).
__global__ void k_sector_reduce_parts(const double* __restrict__ partial, int pmax, const RunBlk* __restrict__ blks,
                                      int nblk, double* out) {
  const int b = (int)((blockIdx.x * (unsigned)blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
  if (b >= nblk) return;  // whole warps leave together
  const int np = blks[b].np;
  double s = 0.0;
  for (int p = lane; p < np; p += 32) s += partial[(size_t)b * pmax + p];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if (lane == 0) out[b] = s;
}


// D_g(b) psi(b) added to (lx, ly) for one connected group; psi(b) is stored at psi[a].
// A real state's groups of several chunks add their fixed-point weights exactly
// and accumulate into lxs (in units of 2^-e).
template <typename T, bool NARROW>
__device__ __forceinline__ unsigned chunk_index(const ExpChunk* W, uint64_t b) {
  unsigned idx = 0;
  if (NARROW) {  // n <= 32: one 32-bit popcount per term
    const uint32_t b32 = (uint32_t)b;
#pragma unroll
    for (int t = 0; t < kChunkTerms; ++t) idx |= ((unsigned)__popc((uint32_t)W->z[t] & b32) & 1u) << t;
  } else {
#pragma unroll
    for (int t = 0; t < kChunkTerms; ++t) idx |= par64s(W->z[t] & b) << t;
  }
  return idx;
}

// Sign pattern of b (n <= 32) against a packed chunk's masks.
__device__ __forceinline__ unsigned real_index(const RealChunk* __restrict__ R, uint32_t b) {
  const uint4 z = __ldg(reinterpret_cast<const uint4*>(R->z));
  return ((unsigned)__popc(z.x & b) & 1u) | (((unsigned)__popc(z.y & b) & 1u) << 1) |
         (((unsigned)__popc(z.z & b) & 1u) << 2) | (((unsigned)__popc(z.w & b) & 1u) << 3);
}

// FP32 partial sums of a complex64 state's H|psi>, folded into the FP64 sum
// after each innermost enumeration loop (at most C(17, 2) = 136 terms at 34
// qubits, 15 to 36 at 24).
struct F32Acc {
  float s = 0.0f;
  __device__ __forceinline__ void add(float w, float v) { s = fmaf(w, v, s); }
  __device__ __forceinline__ void fold(double& lx) {
    lx += (double)s;
    s = 0.0f;
  }
};

template <typename T, bool REALST, bool NARROW>
__device__ __forceinline__ void sector_term(const typename SCx<T>::V* __restrict__ psi,
                                            const ExpChunk* __restrict__ chunks,
                                            const long long* __restrict__ itab, const RealChunk* __restrict__ rch,
                                            int chunk0, int nchunk, uint64_t b, uint64_t a, double& lx, double& ly,
                                            double& lxs, F32Acc& fac) {
  using V = typename SCx<T>::V;
  if (REALST && NARROW && rch) {  // packed real tables
    const T vt = reinterpret_cast<const T*>(psi)[2 * a];
    if (nchunk == 1) {
      const RealChunk* R = rch + chunk0;
      const unsigned idx = real_index(R, (uint32_t)b);
      if (sizeof(T) == 4)  // complex64: FP32 products, folded into the FP64 sum
        fac.add(__ldg(&R->tf[idx]), (float)vt);
      else
        lx = fma(__ldg(&R->t[idx]), (double)vt, lx);
    } else {
      const double v = (double)vt;
      long long is = 0;
      for (int k = 0; k < nchunk; ++k)
        is += __ldg(itab + ((size_t)(chunk0 + k) << kChunkTerms) + real_index(rch + chunk0 + k, (uint32_t)b));
      lxs = fma(__ll2double_rn(is), v, lxs);
    }
    return;
  }
  if (REALST && nchunk > 1) {
    long long is = 0;
    for (int k = 0; k < nchunk; ++k) {
      const ExpChunk* W = chunks + chunk0 + k;
      is += __ldg(itab + ((size_t)(chunk0 + k) << kChunkTerms) + chunk_index<T, NARROW>(W, b));
    }
    lxs = fma(__ll2double_rn(is), (double)reinterpret_cast<const T*>(psi)[2 * a], lxs);
    return;
  }
  double dx = 0.0, dy = 0.0;
  for (int k = 0; k < nchunk; ++k) {
    const ExpChunk* W = chunks + chunk0 + k;
    const double2 d = W->tab[chunk_index<T, NARROW>(W, b)];
    if (k == 0) {
      dx = d.x;
      dy = d.y;
    } else {
      dx += d.x;
      dy += d.y;
    }
  }
  if (REALST) {
    lx = fma(dx, (double)reinterpret_cast<const T*>(psi)[2 * a], lx);
  } else {
    const V v = psi[a];
    lx = fma(dx, (double)v.x, lx);
    lx = fma(-dy, (double)v.y, lx);
    ly = fma(dx, (double)v.y, fma(dy, (double)v.x, ly));
  }
}

// lambda = H psi on the sector members; out[0] = <psi|lambda>, out[1] = <psi|psi>.
// For member c every group that links c to another member flips as many
// occupied as empty alpha (even) and beta (odd) spin orbitals.  Groups of at
// most four flips are reached by enumerating exactly those flips (singles and
// doubles of c) and looking the group up by the rank of its flip set; larger
// groups are tested one by one.
template <typename T, bool REALST, bool NARROW, bool LAMY, bool COMPACT>
__global__ void __launch_bounds__(256) k_sector_hpsi(const typename SCx<T>::V* __restrict__ psi,
                                                     typename SCx<T>::V* __restrict__ lam, SecSpace sp, SecRank rk,
                                                     const SecGroup* __restrict__ large, int nlarge,
                                                     const ExpChunk* __restrict__ chunks, double* partials,
                                                     unsigned* counter, double* out, SecCompact cm) {
  using V = typename SCx<T>::V;
  __shared__ uint32_t C[kBinom][kBinom];
  __shared__ SecSpace ssp;
  fill_binom(C);
  if (threadIdx.x == 0) ssp = sp;
  __syncthreads();
  const uint64_t items = (uint64_t)sp.cnt_e * (uint64_t)sp.cnt_o;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  const uint64_t EVEN = 0x5555555555555555ull, ODD = 0xAAAAAAAAAAAAAAAAull;
  double acc_e = 0.0, acc_n = 0.0;
  for (uint64_t it = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; it < items; it += stride) {
    const uint32_t i32 = (uint32_t)it;
    const uint32_t ie = i32 / ssp.cnt_o, io = i32 - ie * ssp.cnt_o;
    const uint64_t c = unrank(ie, ssp.epos, ssp.ne, ssp.ke, C) | unrank(io, ssp.opos, ssp.no, ssp.ko, C);
    // occupied spin orbitals of each parity as local masks (alpha orbital q is
    // qubit 2q, beta orbital q is qubit 2q + 1), and the empty ones; the loops
    // below visit set bits in ascending order, held in registers
    uint32_t la = 0, lb = 0;  // local alpha / beta strings (compact addressing)
    for (int q = 0; q < ssp.ne; ++q) la |= (uint32_t)((c >> ssp.epos[q]) & 1ull) << q;
    for (int q = 0; q < ssp.no; ++q) lb |= (uint32_t)((c >> ssp.opos[q]) & 1ull) << q;
    const uint32_t va = ((1u << ssp.ne) - 1u) & ~la, vb = ((1u << ssp.no) - 1u) & ~lb;
    double lx = 0.0, ly = 0.0, lxs = 0.0;
    F32Acc fac;
    // one connected group: flip x (qubits), xa / xb (local alpha / beta orbitals)
    auto term = [&](int chunk0, int nchunk, uint64_t x, uint32_t xa, uint32_t xb) {
      const uint64_t b = c ^ x;
      const uint64_t a = COMPACT ? compact_index(cm, la ^ xa, lb ^ xb) : b;
      sector_term<T, REALST, NARROW>(psi, chunks, rk.itab, rk.rch, chunk0, nchunk, b, a, lx, ly, lxs, fac);
    };
    // a lookup-table entry: the group's chunk0 | nchunk << 24, or -1 (no group)
    auto visit = [&](int code, uint64_t x, uint32_t xa, uint32_t xb) {
      if (code >= 0) term(code & 0xFFFFFF, code >> 24, x, xa, xb);
    };
    auto qa = [](int q) { return 1ull << (2 * q); };
    auto qb = [](int q) { return 1ull << (2 * q + 1); };
    visit(rk.diag, 0ull, 0u, 0u);
    const int ne = rk.ne, no = rk.no;
    const int pe = ne * (ne - 1) / 2, po = no * (no - 1) / 2;
    // (complex64: fold the FP32 partial sum after every innermost loop)
    auto fold = [&]() {
      if (sizeof(T) == 4) fac.fold(lx);
    };
    auto low = [](uint32_t m) { return __ffs((int)m) - 1; };  // lowest set bit of m != 0
    for (uint32_t m1 = la; m1; m1 &= m1 - 1) {
      const int o = low(m1);
      for (uint32_t n1 = va; n1; n1 &= n1 - 1) {
        const int v = low(n1);
        visit(__ldg(rk.sa + o * ne + v), qa(o) | qa(v), (1u << o) | (1u << v), 0u);
      }
      fold();
    }
    for (uint32_t m1 = lb; m1; m1 &= m1 - 1) {
      const int o = low(m1);
      for (uint32_t n1 = vb; n1; n1 &= n1 - 1) {
        const int v = low(n1);
        visit(__ldg(rk.sb + o * no + v), qb(o) | qb(v), 0u, (1u << o) | (1u << v));
      }
      fold();
    }
    // same-spin doubles: occupied pairs o1 < o2 (by o2, then o1), empty pairs v1 < v2 likewise
    for (uint32_t m2 = la; m2; m2 &= m2 - 1) {
      const int o2 = low(m2);
      for (uint32_t m1 = la & ((1u << o2) - 1u); m1; m1 &= m1 - 1) {
        const int o1 = low(m1);
        const int rij = o1 + o2 * (o2 - 1) / 2;
        const uint64_t xo = qa(o1) | qa(o2);
        const uint32_t lo = (1u << o1) | (1u << o2);
        for (uint32_t n2 = va; n2; n2 &= n2 - 1) {
          const int v2 = low(n2);
          const int base = rij * pe + v2 * (v2 - 1) / 2;
          for (uint32_t n1 = va & ((1u << v2) - 1u); n1; n1 &= n1 - 1) {
            const int v1 = low(n1);
            visit(__ldg(rk.aa + base + v1), xo | qa(v1) | qa(v2), lo | (1u << v1) | (1u << v2), 0u);
          }
        }
        fold();
      }
    }
    for (uint32_t m2 = lb; m2; m2 &= m2 - 1) {
      const int o2 = low(m2);
      for (uint32_t m1 = lb & ((1u << o2) - 1u); m1; m1 &= m1 - 1) {
        const int o1 = low(m1);
        const int rij = o1 + o2 * (o2 - 1) / 2;
        const uint64_t xo = qb(o1) | qb(o2);
        const uint32_t lo = (1u << o1) | (1u << o2);
        for (uint32_t n2 = vb; n2; n2 &= n2 - 1) {
          const int v2 = low(n2);
          const int base = rij * po + v2 * (v2 - 1) / 2;
          for (uint32_t n1 = vb & ((1u << v2) - 1u); n1; n1 &= n1 - 1) {
            const int v1 = low(n1);
            visit(__ldg(rk.bb + base + v1), xo | qb(v1) | qb(v2), 0u, lo | (1u << v1) | (1u << v2));
          }
        }
        fold();
      }
    }
    // opposite-spin doubles: alpha single (o -> v), then beta single (ob -> vb')
    for (uint32_t m1 = la; m1; m1 &= m1 - 1) {
      const int o = low(m1);
      for (uint32_t n1 = va; n1; n1 &= n1 - 1) {
        const int v = low(n1);
        const int ia = (o * ne + v) * no;
        const uint64_t xa_q = qa(o) | qa(v);
        const uint32_t xa_l = (1u << o) | (1u << v);
        for (uint32_t m2 = lb; m2; m2 &= m2 - 1) {
          const int o2 = low(m2);
          const int iab = (ia + o2) * no;
          for (uint32_t n2 = vb; n2; n2 &= n2 - 1) {
            const int v2 = low(n2);
            visit(__ldg(rk.ab + iab + v2), xa_q | qb(o2) | qb(v2), xa_l, (1u << o2) | (1u << v2));
          }
        }
        fold();
      }
    }
    // groups flipping more than four qubits: test each
    for (int gi = 0; gi < nlarge; ++gi) {
      const SecGroup G = large[gi];
      if (2 * __popcll(c & G.x & EVEN) != G.xe || 2 * __popcll(c & G.x & ODD) != G.xo) continue;
      term(G.chunk0, G.nchunk, G.x, G.xa, G.xb);
      fold();
    }
    const uint64_t self = COMPACT ? it : c;
    fold();  // what is left (a member with no flips)
    if (REALST) lx = fma(lxs, rk.inv_fix, lx);
    if (REALST) {  // real parts only: with LAMY the imaginary slots are lambda's
      const double ux = (double)reinterpret_cast<const T*>(psi)[2 * self];
      acc_e = fma(ux, lx, acc_e);
      acc_n = fma(ux, ux, acc_n);
    } else {
      const V u = psi[self];
      acc_e = fma((double)u.x, lx, fma((double)u.y, ly, acc_e));
      acc_n = fma((double)u.x, (double)u.x, fma((double)u.y, (double)u.y, acc_n));
    }
    if (LAMY) {  // lambda's real part into psi's imaginary slot (real states)
      reinterpret_cast<T*>(lam)[2 * self + 1] = (T)lx;
    } else if (lam) {
      V w;
      w.x = (T)lx;
      w.y = (T)ly;
      lam[self] = w;
    }
  }
  // deterministic two-value grid reduction
  __shared__ bool last;
  const double b0 = block_sum_s(acc_e);
  const double b1 = block_sum_s(acc_n);
  if (threadIdx.x == 0) {
    partials[2 * blockIdx.x] = b0;
    partials[2 * blockIdx.x + 1] = b1;
    __threadfence();
    last = (atomicAdd(counter, 1u) == gridDim.x - 1);
  }
  __syncthreads();
  if (last) {
    __threadfence();
    double s0 = 0.0, s1 = 0.0;
    for (unsigned i = threadIdx.x; i < gridDim.x; i += blockDim.x) {
      s0 += __ldcg(partials + 2 * i);
      s1 += __ldcg(partials + 2 * i + 1);
    }
    s0 = block_sum_s(s0);
    s1 = block_sum_s(s1);
    if (threadIdx.x == 0) {
      out[0] = s0;
      out[1] = s1;
      *counter = 0u;
    }
  }
}

// ---------------------------------------------------------------------------
// Sector H|psi> through the direct tables (SecDirect), compact layout, real
// state with lambda packed into psi's imaginary slots.  Per member: the
// prefix-parity bits PP_c at every qubit, then every single and double flip of
// c -- each costs one table weight, its sign from four (two) PP bits, the
// partner's rank and one multiply-add.  The diagonal and the singles' number-
// operator parts are summed exactly in fixed point.

// The r-th k-subset (colex order) of positions 0..m-1 as a bit mask.
__device__ __forceinline__ uint32_t unrank_mask(uint32_t r, int m, int k, const uint32_t (*C)[kBinom]) {
  uint32_t bits = 0;
  for (int j = m - 1; j >= 0 && k > 0; --j) {
    const uint32_t c = C[j][k];
    if (r >= c) {
      bits |= 1u << j;
      r -= c;
      --k;
    }
  }
  return bits;
}

// Bit q of x (q < 16) to bit 2q.
__device__ __forceinline__ uint32_t spread16(uint32_t x) {
  x = (x | (x << 8)) & 0x00FF00FFu;
  x = (x | (x << 4)) & 0x0F0F0F0Fu;
  x = (x | (x << 2)) & 0x33333333u;
  x = (x | (x << 1)) & 0x55555555u;
  return x;
}

// Bit 2q of x to bit q.
__device__ __forceinline__ uint32_t gather_even(uint32_t x) {
  x &= 0x55555555u;
  x = (x | (x >> 1)) & 0x33333333u;
  x = (x | (x >> 2)) & 0x0F0F0F0Fu;
  x = (x | (x >> 4)) & 0x00FF00FFu;
  x = (x | (x >> 8)) & 0x0000FFFFu;
  return x;
}

// w with its sign flipped when s (0 or 1) is set.
__device__ __forceinline__ double flip_sign(double w, uint32_t s) {
  return __longlong_as_double(__double_as_longlong(w) ^ ((long long)s << 63));
}
__device__ __forceinline__ float flip_sign(float w, uint32_t s) {
  return __int_as_float(__float_as_int(w) ^ (int)(s << 31));
}

// Pair products of one member: FP64 multiply-adds into the member's sum
// (complex128), or FP32 ones added after each innermost loop (at most C(16, 2)
// products) into a float-pair total that is converted to FP64 once (complex64).
template <typename T> struct PairAcc {
  float s = 0.0f;
  __device__ __forceinline__ void add(float w, float v, double&) { s = fmaf(w, v, s); }
  // s added into the float-pair total (hi, lo) by a TwoSum: no FP64 operation
  __device__ __forceinline__ void fold_into(float& hi, float& lo) {
    const float t = __fadd_rn(hi, s);
    const float bp = __fsub_rn(t, hi);
    const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(t, bp)), __fsub_rn(s, bp));
    const float l = __fadd_rn(lo, err);
    hi = __fadd_rn(t, l);
    lo = __fsub_rn(l, __fsub_rn(hi, t));
    s = 0.0f;
  }
};
template <> struct PairAcc<double> {
  __device__ __forceinline__ void add(double w, double v, double& lx) { lx = fma(w, v, lx); }
  __device__ __forceinline__ void fold_into(float&, float&) {}
};

// Double-single pair products (complex128, QF_HPSI_DS): a weight and an amplitude
// each as a float pair hi + lo (about 48 significant bits); the product keeps the
// exact error of hi * hi and both cross terms, the float-pair sum takes it through
// an error-free TwoSum, and after each innermost loop (at most C(16, 2)^2 / 16
// products) the sum is added into the member's double-single total, which is
// converted to FP64 once.  The rounded operations are explicit so that no
// multiply is fused into the TwoSum.
struct DsAcc {
  float sh = 0.0f, sl = 0.0f;
  __device__ __forceinline__ void add(float2 w, float2 v) {
    const float ph = __fmul_rn(w.x, v.x);
    float pl = fmaf(w.x, v.x, -ph);
    pl = fmaf(w.x, v.y, pl);
    pl = fmaf(w.y, v.x, pl);
    const float s = __fadd_rn(sh, ph);
    const float bp = __fsub_rn(s, sh);
    const float err = __fadd_rn(__fsub_rn(sh, __fsub_rn(s, bp)), __fsub_rn(ph, bp));
    sl = __fadd_rn(sl, __fadd_rn(err, pl));
    sh = s;
  }
  __device__ __forceinline__ void fold(double& lx) {
    lx += (double)sh + (double)sl;
    sh = 0.0f;
    sl = 0.0f;
  }
  // this sum added into o as a double-single value (TwoSum of the high parts, the
  // low parts and the error summed, one renormalisation): no FP64 operation
  __device__ __forceinline__ void fold_into(DsAcc& o) {
    const float s = __fadd_rn(o.sh, sh);
    const float bp = __fsub_rn(s, o.sh);
    const float err = __fadd_rn(__fsub_rn(o.sh, __fsub_rn(s, bp)), __fsub_rn(sh, bp));
    const float lo = __fadd_rn(__fadd_rn(o.sl, sl), err);
    const float h = __fadd_rn(s, lo);
    o.sl = __fsub_rn(lo, __fsub_rn(h, s));
    o.sh = h;
    sh = 0.0f;
    sl = 0.0f;
  }
};
__device__ __forceinline__ float2 flip_sign2(float2 w, uint32_t s) {
  return make_float2(flip_sign(w.x, s), flip_sign(w.y, s));
}

// (hi, lo) float split of every member's real amplitude (packed state: psi at 2 m).
// dss: the state is already in double-single form, (psi hi, psi lo, lam hi, lam
// lo) floats per member; the split is copied out and psid[m] gets psi as a double.
__global__ void k_split_real(const double* __restrict__ st, float2* __restrict__ out, double* __restrict__ psid,
                             uint64_t members, bool dss) {
  for (uint64_t m = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; m < members;
       m += (uint64_t)gridDim.x * blockDim.x) {
    if (dss) {
      const float2 v = __ldcg(reinterpret_cast<const float2*>(st) + 2 * m);
      out[m] = v;
      psid[m] = (double)v.x + (double)v.y;
    } else {
      const double v = st[2 * m];
      const float hi = __double2float_rn(v);
      out[m] = make_float2(hi, __double2float_rn(v - (double)hi));
    }
  }
}

// lambda of one member (it: its compact index) through the direct tables:
// the diagonal, the singles (fixed-point weights), then the opposite- and
// same-spin doubles as pair products.  amp(idx): psi of member idx as a double
// (the diagonal and singles); pair(idx): its pair-product operand -- T in FP64
// or FP32, the (hi, lo) float split with DS.  bl: this thread's beta-single list,
// entry k at bl[k * BSTRIDE].
template <typename T, bool DS, int BSTRIDE, typename AmpF, typename PairF>
__device__ __forceinline__ double direct_member(uint32_t it, const SecDirect& d, uint32_t cnt_o, int ke, int ko,
                                                const uint16_t* __restrict__ ra, const uint16_t* __restrict__ rb,
                                                const uint32_t (*C)[kBinom], uint32_t* bl, AmpF amp, PairF pair) {
  const int n = d.n, ne = d.ne, no = d.no;
  const int pe = ne * (ne - 1) / 2, po = no * (no - 1) / 2;
  const T* wab = reinterpret_cast<const T*>(sizeof(T) == 8 ? (const void*)d.wab : (const void*)d.fab);
  const T* waa = reinterpret_cast<const T*>(sizeof(T) == 8 ? (const void*)d.waa : (const void*)d.faa);
  const T* wbb = reinterpret_cast<const T*>(sizeof(T) == 8 ? (const void*)d.wbb : (const void*)d.fbb);
  const uint32_t ie = it / cnt_o, io = it - ie * cnt_o;
  const uint32_t la = unrank_mask(ie, ne, ke, C), lb = unrank_mask(io, no, ko, C);
  const uint32_t c = spread16(la) | (spread16(lb) << 1);  // the member in qubit order
  uint32_t p = c;  // prefix parities: bit q = parity of c's bits below q
  p ^= p << 1;
  p ^= p << 2;
  p ^= p << 4;
  p ^= p << 8;
  p ^= p << 16;
  p <<= 1;
  const uint32_t ppa = gather_even(p), ppb = gather_even(p >> 1);
  const uint32_t va = ((1u << ne) - 1u) & ~la, vb = ((1u << no) - 1u) & ~lb;
  const size_t rowself = (size_t)ie * cnt_o;
  double lx = 0.0, lxs = 0.0;  // lxs: fixed-point weights times psi (units of 2^-e)
  PairAcc<T> pa, pb;  // two accumulators, so that two chains are in flight
  DsAcc da, db, dt;   // dt: the member's float-pair total of the pair products, converted to FP64 once
  // x = 0: K + sum U[r] + sum V[r][s] over occupied r < s
  long long dsum = __ldg(d.dg);
  for (uint32_t m = c; m; m &= m - 1) {
    const int r = __ffs((int)m) - 1;
    dsum += __ldg(d.dg + 1 + r);
    const long long* vr = d.dg + 1 + n + r * n - 1;
    for (uint32_t m2 = m & (m - 1); m2; m2 &= m2 - 1) dsum += __ldg(vr + __ffs((int)m2));
  }
  lxs = fma(__ll2double_rn(dsum), amp(it), lxs);
  // singles: A + sum of B[r] over c's occupied qubits other than the one it gives up
  for (uint32_t m1 = la; m1; m1 &= m1 - 1) {
    const int o = __ffs((int)m1) - 1;
    const uint32_t rest = c & ~(1u << (2 * o));
    for (uint32_t n1 = va; n1; n1 &= n1 - 1) {
      const int v = __ffs((int)n1) - 1;
      const long long* row = d.s1a + (size_t)(o * ne + v) * (n + 1);
      long long w = __ldg(row);
      for (uint32_t m2 = rest; m2; m2 &= m2 - 1) w += __ldg(row + __ffs((int)m2));
      if (((ppa >> o) ^ (ppa >> v)) & 1u) w = -w;
      const size_t idx = (size_t)__ldg(ra + (la ^ (1u << o) ^ (1u << v))) * cnt_o + io;
      lxs = fma(__ll2double_rn(w), amp(idx), lxs);
    }
  }
  for (uint32_t m1 = lb; m1; m1 &= m1 - 1) {
    const int o = __ffs((int)m1) - 1;
    const uint32_t rest = c & ~(1u << (2 * o + 1));
    for (uint32_t n1 = vb; n1; n1 &= n1 - 1) {
      const int v = __ffs((int)n1) - 1;
      const long long* row = d.s1b + (size_t)(o * no + v) * (n + 1);
      long long w = __ldg(row);
      for (uint32_t m2 = rest; m2; m2 &= m2 - 1) w += __ldg(row + __ffs((int)m2));
      if (((ppb >> o) ^ (ppb >> v)) & 1u) w = -w;
      const size_t idx = rowself + __ldg(rb + (lb ^ (1u << o) ^ (1u << v)));
      lxs = fma(__ll2double_rn(w), amp(idx), lxs);
    }
  }
  // opposite-spin doubles: alpha o -> v, beta o2 -> v2; the member's beta singles
  // are listed once and reused under each of its alpha singles
  int nbs = 0;
  for (uint32_t m2 = lb; m2; m2 &= m2 - 1) {
    const int o2 = __ffs((int)m2) - 1;
    const uint32_t lbo = lb ^ (1u << o2);
    const uint32_t so = (ppb >> o2) & 1u;
    for (uint32_t n2 = vb; n2; n2 &= n2 - 1) {
      const int v2 = __ffs((int)n2) - 1;
      bl[BSTRIDE * nbs++] = (uint32_t)__ldg(rb + (lbo | (1u << v2))) | ((uint32_t)(o2 * no + v2) << 14) |
                            ((so ^ ((ppb >> v2) & 1u)) << 31);
    }
  }
  for (uint32_t m1 = la; m1; m1 &= m1 - 1) {
    const int o = __ffs((int)m1) - 1;
    for (uint32_t n1 = va; n1; n1 &= n1 - 1) {
      const int v = __ffs((int)n1) - 1;
      const uint32_t sa = ((ppa >> o) ^ (ppa >> v)) & 1u;
      const size_t rowa = (size_t)__ldg(ra + (la ^ (1u << o) ^ (1u << v))) * cnt_o;
      const size_t wo = (size_t)(o * ne + v) * (no * no);
      const T* wrow = wab + wo;
      const float2* drow = d.dab + wo;
      if constexpr (DS) {
        // two independent accumulators (alternate entries), so that two TwoSum
        // chains are in flight, and four entries' loads issued together
        int k = 0;
        for (; k + 3 < nbs; k += 4) {
          const uint32_t e0 = bl[BSTRIDE * k], e1 = bl[BSTRIDE * (k + 1)];
          const uint32_t e2 = bl[BSTRIDE * (k + 2)], e3 = bl[BSTRIDE * (k + 3)];
          const float2 w0 = __ldg(drow + ((e0 >> 14) & 0xFFu)), w1 = __ldg(drow + ((e1 >> 14) & 0xFFu));
          const float2 w2 = __ldg(drow + ((e2 >> 14) & 0xFFu)), w3 = __ldg(drow + ((e3 >> 14) & 0xFFu));
          const float2 v0 = pair(rowa + (e0 & 0x3FFFu)), v1 = pair(rowa + (e1 & 0x3FFFu));
          const float2 v2 = pair(rowa + (e2 & 0x3FFFu)), v3 = pair(rowa + (e3 & 0x3FFFu));
          da.add(flip_sign2(w0, sa ^ (e0 >> 31)), v0);
          db.add(flip_sign2(w1, sa ^ (e1 >> 31)), v1);
          da.add(flip_sign2(w2, sa ^ (e2 >> 31)), v2);
          db.add(flip_sign2(w3, sa ^ (e3 >> 31)), v3);
        }
        for (; k + 1 < nbs; k += 2) {
          const uint32_t e0 = bl[BSTRIDE * k], e1 = bl[BSTRIDE * (k + 1)];
          const float2 w0 = __ldg(drow + ((e0 >> 14) & 0xFFu)), w1 = __ldg(drow + ((e1 >> 14) & 0xFFu));
          const float2 v0 = pair(rowa + (e0 & 0x3FFFu)), v1 = pair(rowa + (e1 & 0x3FFFu));
          da.add(flip_sign2(w0, sa ^ (e0 >> 31)), v0);
          db.add(flip_sign2(w1, sa ^ (e1 >> 31)), v1);
        }
        if (k < nbs) {
          const uint32_t e = bl[BSTRIDE * k];
          da.add(flip_sign2(__ldg(drow + ((e >> 14) & 0xFFu)), sa ^ (e >> 31)), pair(rowa + (e & 0x3FFFu)));
        }
        da.fold_into(dt);
        db.fold_into(dt);
      } else {
        int k = 0;
        for (; k + 3 < nbs; k += 4) {
          const uint32_t e0 = bl[BSTRIDE * k], e1 = bl[BSTRIDE * (k + 1)];
          const uint32_t e2 = bl[BSTRIDE * (k + 2)], e3 = bl[BSTRIDE * (k + 3)];
          const T w0 = __ldg(wrow + ((e0 >> 14) & 0xFFu)), w1 = __ldg(wrow + ((e1 >> 14) & 0xFFu));
          const T w2 = __ldg(wrow + ((e2 >> 14) & 0xFFu)), w3 = __ldg(wrow + ((e3 >> 14) & 0xFFu));
          const T v0 = pair(rowa + (e0 & 0x3FFFu)), v1 = pair(rowa + (e1 & 0x3FFFu));
          const T v2 = pair(rowa + (e2 & 0x3FFFu)), v3 = pair(rowa + (e3 & 0x3FFFu));
          pa.add(flip_sign(w0, sa ^ (e0 >> 31)), v0, lx);
          pb.add(flip_sign(w1, sa ^ (e1 >> 31)), v1, lx);
          pa.add(flip_sign(w2, sa ^ (e2 >> 31)), v2, lx);
          pb.add(flip_sign(w3, sa ^ (e3 >> 31)), v3, lx);
        }
        for (; k + 1 < nbs; k += 2) {
          const uint32_t e0 = bl[BSTRIDE * k], e1 = bl[BSTRIDE * (k + 1)];
          const T w0 = __ldg(wrow + ((e0 >> 14) & 0xFFu)), w1 = __ldg(wrow + ((e1 >> 14) & 0xFFu));
          const T v0 = pair(rowa + (e0 & 0x3FFFu)), v1 = pair(rowa + (e1 & 0x3FFFu));
          pa.add(flip_sign(w0, sa ^ (e0 >> 31)), v0, lx);
          pb.add(flip_sign(w1, sa ^ (e1 >> 31)), v1, lx);
        }
        if (k < nbs) {
          const uint32_t e = bl[BSTRIDE * k];
          pa.add(flip_sign(__ldg(wrow + ((e >> 14) & 0xFFu)), sa ^ (e >> 31)), pair(rowa + (e & 0x3FFFu)), lx);
        }
        pa.fold_into(dt.sh, dt.sl);
        pb.fold_into(dt.sh, dt.sl);
      }
    }
  }
  // same-spin doubles: occupied o1 < o2 -> empty v1 < v2
  for (uint32_t m2 = la; m2; m2 &= m2 - 1) {
    const int o2 = __ffs((int)m2) - 1;
    for (uint32_t m1 = la & ((1u << o2) - 1u); m1; m1 &= m1 - 1) {
      const int o1 = __ffs((int)m1) - 1;
      const uint32_t so = ((ppa >> o1) ^ (ppa >> o2)) & 1u;
      const uint32_t lao = la ^ (1u << o1) ^ (1u << o2);
      const size_t wo = (size_t)(o1 + o2 * (o2 - 1) / 2) * pe;
      for (uint32_t n2 = va; n2; n2 &= n2 - 1) {
        const int v2 = __ffs((int)n2) - 1;
        const uint32_t s2 = so ^ ((ppa >> v2) & 1u);
        const size_t w2 = wo + v2 * (v2 - 1) / 2;
        const uint32_t lav = lao | (1u << v2);
        // two entries per round (the second into db / pb), so that two chains and
        // their loads are in flight
        for (uint32_t n1 = va & ((1u << v2) - 1u); n1;) {
          const int v1 = __ffs((int)n1) - 1;
          n1 &= n1 - 1;
          const size_t idx = (size_t)__ldg(ra + (lav | (1u << v1))) * cnt_o + io;
          const uint32_t sg = s2 ^ ((ppa >> v1) & 1u);
          if (n1) {
            const int u1 = __ffs((int)n1) - 1;
            n1 &= n1 - 1;
            const size_t jdx = (size_t)__ldg(ra + (lav | (1u << u1))) * cnt_o + io;
            const uint32_t tg = s2 ^ ((ppa >> u1) & 1u);
            if constexpr (DS)
              db.add(flip_sign2(__ldg(d.daa + w2 + u1), tg), pair(jdx));
            else
              pb.add(flip_sign(__ldg(waa + w2 + u1), tg), pair(jdx), lx);
          }
          if constexpr (DS)
            da.add(flip_sign2(__ldg(d.daa + w2 + v1), sg), pair(idx));
          else
            pa.add(flip_sign(__ldg(waa + w2 + v1), sg), pair(idx), lx);
        }
      }
      if constexpr (DS) {
        da.fold_into(dt);
        db.fold_into(dt);
      } else {
        pa.fold_into(dt.sh, dt.sl);
        pb.fold_into(dt.sh, dt.sl);
      }
    }
  }
  for (uint32_t m2 = lb; m2; m2 &= m2 - 1) {
    const int o2 = __ffs((int)m2) - 1;
    for (uint32_t m1 = lb & ((1u << o2) - 1u); m1; m1 &= m1 - 1) {
      const int o1 = __ffs((int)m1) - 1;
      const uint32_t so = ((ppb >> o1) ^ (ppb >> o2)) & 1u;
      const uint32_t lbo = lb ^ (1u << o1) ^ (1u << o2);
      const size_t wo = (size_t)(o1 + o2 * (o2 - 1) / 2) * po;
      for (uint32_t n2 = vb; n2; n2 &= n2 - 1) {
        const int v2 = __ffs((int)n2) - 1;
        const uint32_t s2 = so ^ ((ppb >> v2) & 1u);
        const size_t w2 = wo + v2 * (v2 - 1) / 2;
        const uint32_t lbv = lbo | (1u << v2);
        for (uint32_t n1 = vb & ((1u << v2) - 1u); n1;) {
          const int v1 = __ffs((int)n1) - 1;
          n1 &= n1 - 1;
          const size_t idx = rowself + __ldg(rb + (lbv | (1u << v1)));
          const uint32_t sg = s2 ^ ((ppb >> v1) & 1u);
          if (n1) {
            const int u1 = __ffs((int)n1) - 1;
            n1 &= n1 - 1;
            const size_t jdx = rowself + __ldg(rb + (lbv | (1u << u1)));
            const uint32_t tg = s2 ^ ((ppb >> u1) & 1u);
            if constexpr (DS)
              db.add(flip_sign2(__ldg(d.dbb + w2 + u1), tg), pair(jdx));
            else
              pb.add(flip_sign(__ldg(wbb + w2 + u1), tg), pair(jdx), lx);
          }
          if constexpr (DS)
            da.add(flip_sign2(__ldg(d.dbb + w2 + v1), sg), pair(idx));
          else
            pa.add(flip_sign(__ldg(wbb + w2 + v1), sg), pair(idx), lx);
        }
      }
      if constexpr (DS) {
        da.fold_into(dt);
        db.fold_into(dt);
      } else {
        pa.fold_into(dt.sh, dt.sl);
        pb.fold_into(dt.sh, dt.sl);
      }
    }
  }
  dt.fold(lx);  // the pair products' float-pair total (zero for FP64 products)
  return fma(lxs, d.inv_fix, lx);
}

template <typename T, bool DS>
__global__ void __launch_bounds__(256, 4) k_sector_hpsi_direct(T* st, SecDirect d, uint32_t cnt_e, uint32_t cnt_o,
                                                            int ke, int ko, const uint16_t* __restrict__ ra,
                                                            const uint16_t* __restrict__ rb, double* partials,
                                                            unsigned* counter, double* out,
                                                            const float2* __restrict__ split,
                                                            const double* __restrict__ psid, bool dss) {
  __shared__ uint32_t C[kBinom][kBinom];
  // each thread's beta singles (entry k of thread t at bsl[k * 256 + t]): the
  // flipped string's rank | weight column o2 * no + v2 << 14 | sign bit << 31
  extern __shared__ uint32_t bsl[];
  fill_binom(C);
  __syncthreads();
  const T* ps = st;  // psi of member m at ps[2 m]; lambda goes to st[2 m + 1]
  // psi of member m as a double: pd[pst * m] (double-single state layout: psid, from the split)
  const double* pd = (DS && dss) ? psid : reinterpret_cast<const double*>(ps);
  const int pst = (DS && dss) ? 1 : 2;
  auto amp = [&](size_t m) -> double { return (sizeof(T) == 8) ? pd[pst * m] : (double)ps[2 * m]; };
  auto pair_op = [&](size_t m) {
    if constexpr (DS)
      return __ldg(split + m);
    else
      return ps[2 * m];
  };
  const uint64_t items = (uint64_t)cnt_e * cnt_o;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  double acc_e = 0.0, acc_n = 0.0;
  for (uint64_t it = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; it < items; it += stride) {
    const double self = amp(it);
    const double lx = direct_member<T, DS, 256>((uint32_t)it, d, cnt_o, ke, ko, ra, rb, C, bsl + threadIdx.x, amp,
                                                pair_op);
    acc_e = fma(self, lx, acc_e);
    acc_n = fma(self, self, acc_n);
    if (DS && dss)
      reinterpret_cast<float2*>(st)[2 * (size_t)it + 1] = ds_of(lx);
    else
      st[2 * (size_t)it + 1] = (T)lx;
  }
  // deterministic two-value grid reduction
  __shared__ bool last;
  const double b0 = block_sum_s(acc_e);
  const double b1 = block_sum_s(acc_n);
  if (threadIdx.x == 0) {
    partials[2 * blockIdx.x] = b0;
    partials[2 * blockIdx.x + 1] = b1;
    __threadfence();
    last = (atomicAdd(counter, 1u) == gridDim.x - 1);
  }
  __syncthreads();
  if (last) {
    __threadfence();
    double s0 = 0.0, s1 = 0.0;
    for (unsigned i = threadIdx.x; i < gridDim.x; i += blockDim.x) {
      s0 += __ldcg(partials + 2 * i);
      s1 += __ldcg(partials + 2 * i + 1);
    }
    s0 = block_sum_s(s0);
    s1 = block_sum_s(s1);
    if (threadIdx.x == 0) {
      out[0] = s0;
      out[1] = s1;
      *counter = 0u;
    }
  }
}

// Small systems, several requests per launch (SmallEval): CTA r evaluates request
// r alone.  Its compact state (psi, then lambda: members real values each) and
// the H psi step's beta-single lists live in shared memory; the block
// geometries, tables and rank tables are shared by every CTA and stay in L1/L2.
constexpr int kSmallThreads = 256;

// The two compact indices and the sign class of item `it` of block B (the item's
// outside string in colex order, as the full-layout sweep enumerates it).
__device__ __forceinline__ void small_item(const SecBlk& B, uint32_t it, const uint32_t (*C)[kBinom],
                                           const uint16_t* __restrict__ ra, const uint16_t* __restrict__ rb,
                                           uint32_t cnt_o, uint32_t* i0, uint32_t* i1, unsigned* cls) {
  const uint32_t ie = it / B.cnt_o, io = it - ie * B.cnt_o;
  const uint64_t base = unrank(ie, B.epos, B.ne, B.ke, C) | unrank(io, B.opos, B.no, B.ko, C);
  unsigned c = 0;
  if (B.nzc > 0) c = par64s(B.zc[0] & base);
  if (B.nzc > 1) c |= par64s(B.zc[1] & base) << 1;
  const uint32_t q0 = (uint32_t)(base | B.pat[0]), q1 = (uint32_t)(base | B.pat[1]);
  *i0 = (uint32_t)__ldg(ra + gather_even(q0)) * cnt_o + __ldg(rb + gather_even(q0 >> 1));
  *i1 = (uint32_t)__ldg(ra + gather_even(q1)) * cnt_o + __ldg(rb + gather_even(q1 >> 1));
  *cls = c;
}

template <typename T>
__global__ void __launch_bounds__(kSmallThreads, 2) k_small_eval(SmallEval a) {
  extern __shared__ __align__(16) unsigned char dsm[];
  __shared__ uint32_t C[kBinom][kBinom];
  const int tid = threadIdx.x;
  const uint32_t M = a.cnt_e * a.cnt_o;
  T* ps = reinterpret_cast<T*>(dsm);
  T* lm = ps + M;
  uint32_t* bsl = reinterpret_cast<uint32_t*>(dsm + align16(2 * (size_t)M * sizeof(T)));
  const T* cf = static_cast<const T*>(a.coef) + (size_t)blockIdx.x * a.nblk * kSmallCoef;
  double* out = a.out + (size_t)blockIdx.x * (a.nblk + 2);
  fill_binom(C);
  for (uint32_t m = tid; m < M; m += kSmallThreads) ps[m] = (m == a.c0) ? T(1) : T(0);
  __syncthreads();
  // forward: psi <- psi + (M - I) psi on every item of each block in turn
  for (int b = 0; b < a.nblk; ++b) {
    const SecBlk& B = a.blks[b];
    const T* mf = cf + (size_t)b * kSmallCoef;
    const uint32_t items = B.cnt_e * B.cnt_o;
    for (uint32_t it = tid; it < items; it += kSmallThreads) {
      uint32_t i0, i1;
      unsigned cls;
      small_item(B, it, C, a.ra, a.rb, a.cnt_o, &i0, &i1, &cls);
      const T* m = mf + 4 * cls;
      const T v0 = ps[i0], v1 = ps[i1];
      ps[i0] = fma(m[0], v0, fma(m[1], v1, v0));
      ps[i1] = fma(m[2], v0, fma(m[3], v1, v1));
    }
    __syncthreads();
  }
  // lambda = H psi with <psi|lambda> and <psi|psi>
  double acc_e = 0.0, acc_n = 0.0;
  auto amp = [&](size_t m) -> double { return (double)ps[m]; };
  auto pair_op = [&](size_t m) { return ps[m]; };
  for (uint32_t m = tid; m < M; m += kSmallThreads) {
    const double self = (double)ps[m];
    const double lx = direct_member<T, false, kSmallThreads>(m, a.d, a.cnt_o, a.ke, a.ko, a.ra, a.rb, C, bsl + tid,
                                                             amp, pair_op);
    lm[m] = (T)lx;
    acc_e = fma(self, lx, acc_e);
    acc_n = fma(self, self, acc_n);
  }
  acc_e = block_sum_s(acc_e);
  acc_n = block_sum_s(acc_n);
  if (tid == 0) {
    out[a.nblk] = acc_e;
    out[a.nblk + 1] = acc_n;
  }
  __syncthreads();
  // reverse: block b's overlap Im <lambda|Q_b|psi> = q01 (lambda0 psi1 - lambda1 psi0)
  // summed over its items, then psi and lambda un-rotated by its inverse
  for (int b = a.nblk - 1; b >= 0; --b) {
    const SecBlk& B = a.blks[b];
    const T* mi = cf + (size_t)b * kSmallCoef + 16;
    const T* q = cf + (size_t)b * kSmallCoef + 32;
    const uint32_t items = B.cnt_e * B.cnt_o;
    double acc = 0.0;
    for (uint32_t it = tid; it < items; it += kSmallThreads) {
      uint32_t i0, i1;
      unsigned cls;
      small_item(B, it, C, a.ra, a.rb, a.cnt_o, &i0, &i1, &cls);
      const T* m = mi + 4 * cls;
      const T p0 = ps[i0], p1 = ps[i1], w0 = lm[i0], w1 = lm[i1];
      acc += (double)(q[cls] * fma(w0, p1, -w1 * p0));
      ps[i0] = fma(m[0], p0, fma(m[1], p1, p0));
      ps[i1] = fma(m[2], p0, fma(m[3], p1, p1));
      lm[i0] = fma(m[0], w0, fma(m[1], w1, w0));
      lm[i1] = fma(m[2], w0, fma(m[3], w1, w1));
    }
    acc = block_sum_s(acc);  // its first barrier also ends this block's updates
    if (tid == 0) out[b] = acc;
  }
}

}  // namespace

// Grid of the cooperative sweep: about one item per thread for a typical block,
// at most one CTA per SM (all CTAs must be resident at once; a 1024-thread CTA
// under __launch_bounds__ always fits one per SM).
int sector_sweep_grid(uint64_t typical_items) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const uint64_t want = (typical_items + kSweepThreads - 1) / kSweepThreads;
  return (int)std::max<uint64_t>(1, std::min<uint64_t>(want, (uint64_t)std::max(1, sms)));
}

template <bool REALST, typename T>
static cudaError_t sweep_t(void* psi, const SecBlk* blks, int nblk, unsigned* bar, int grid, cudaStream_t s) {
  using V = typename SCx<T>::V;
  V* p = static_cast<V*>(psi);
  void* args[] = {&p, &blks, &nblk, &bar};
  return cudaLaunchCooperativeKernel((const void*)k_sector_sweep<REALST, T>, dim3(grid), dim3(kSweepThreads), args,
                                     0, s);
}

cudaError_t launch_wait_selftest(unsigned* words, double limit_s, cudaStream_t s) {
  k_wait_selftest<<<1, 32, 0, s>>>(words, (uint64_t)(limit_s * 1e9));
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_sector_sweep(void* psi, qf_dtype dt, bool realst, const SecBlk* blks, int nblk, unsigned* bar,
                                int grid, cudaStream_t s) {
  if (nblk <= 0) return cudaSuccess;
  const int prof_slot_ = prof_pre(QF_K_SPARSE, s);
  cudaError_t e = cudaMemsetAsync(bar, 0, 3 * sizeof(unsigned), s);
  if (e == cudaSuccess) {
    if (dt == QF_C128)
      e = realst ? sweep_t<true, double>(psi, blks, nblk, bar, grid, s)
                 : sweep_t<false, double>(psi, blks, nblk, bar, grid, s);
    else
      e = realst ? sweep_t<true, float>(psi, blks, nblk, bar, grid, s)
                 : sweep_t<false, float>(psi, blks, nblk, bar, grid, s);
  }
  count_launch();
  prof_post(prof_slot_, s);
  return e;
}

// Dynamic shared memory a k_sector_run instantiation may take: the opt-in
// maximum less its static shared memory (binomial tables, descriptors, overlaps).
template <int MODE, typename T>
static size_t run_smem_max() {
  static const int v = [] {  // thread-safe one-time initialisation
    int dev = 0, bytes = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&bytes, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaFuncAttributes fa{};
    if (cudaFuncGetAttributes(&fa, k_sector_run<MODE, T>) != cudaSuccess) {
      cudaGetLastError();
      return 0;
    }
    return std::max(0, bytes - (int)fa.sharedSizeBytes - 256);
  }();
  return (size_t)v;
}

template <int MODE, typename T>
static size_t run_smem_bytes(uint32_t maxsize) {
  constexpr size_t idx = MODE == 4 ? 0 : sizeof(uint32_t);
  const size_t amp = align16((run_member_bytes<MODE, T>() - idx) * maxsize);
  return align16(amp + idx * maxsize);
}

template <int MODE, typename T>
static uint32_t run_capacity_t() {
  const size_t avail = run_smem_max<MODE, T>();
  const size_t fixed = 64;
  return avail > fixed ? (uint32_t)((avail - fixed) / run_member_bytes<MODE, T>()) : 0u;
}

uint32_t sector_run_capacity(qf_dtype dt, bool adj, bool realst, bool logged) {
  const int mode = !adj ? 0 : !realst ? 2 : logged ? 3 : 1;
  if (dt == QF_C128)
    return mode == 0 ? run_capacity_t<0, double>() : mode == 1 ? run_capacity_t<1, double>()
         : mode == 2 ? run_capacity_t<2, double>() : run_capacity_t<3, double>();
  return mode == 0 ? run_capacity_t<0, float>() : mode == 1 ? run_capacity_t<1, float>()
       : mode == 2 ? run_capacity_t<2, float>() : run_capacity_t<3, float>();
}

template <int MODE, typename T, bool DSW = false>
static cudaError_t runs_t(void* psi, void* lam, const RunInfo* runs, int nruns, const RunPart* parts,
                          const RunBlk* blks, double* partial, int pmax, const SecCompact& cm, void* log,
                          const uint16_t* strs, const uint32_t* map, bool dss, cudaStream_t s) {
  static_assert(!DSW || ((MODE == 0 || MODE == 3) && sizeof(T) == 8), "double-single sweeps: complex128 forward "
                                                                      "and logged reverse");
  if (DSW && !map) return cudaErrorInvalidValue;  // the double-single path is the mapped step loop
  using V = typename SCx<T>::V;
  // the mapped step loop runs wide CTAs (not the FP64 logged reverse: at 64
  // registers four of its wide CTAs would not fit an SM)
  constexpr bool kWide = MODE == 0 || (MODE == 3 && (DSW || sizeof(T) == 4));
  const bool wide = kWide && map != nullptr;
  static std::once_flag once;  // allow the opt-in shared memory size, once per process
  static cudaError_t attr = cudaSuccess;
  std::call_once(once, [] {
    const int bytes = (int)run_smem_max<MODE, T>();
    if (!DSW) attr = cudaFuncSetAttribute(k_sector_run<MODE, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if constexpr (kWide)
      if (attr == cudaSuccess)
        attr = cudaFuncSetAttribute(k_sector_run_wide<MODE, T, DSW>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    bytes);
  });
  if (attr != cudaSuccess) return attr;
  for (int r = 0; r < nruns; ++r) {
    const RunInfo& R = runs[MODE != 0 ? nruns - 1 - r : r];
    const size_t smem = run_smem_bytes<MODE, T>(R.maxsize);
    if (smem > run_smem_max<MODE, T>() || R.b1 - R.b0 > kRunMaxBlocks || R.nparts <= 0) return cudaErrorInvalidValue;
    if constexpr (kWide) {
      if (wide) {  // programmatic dependent launch: its table prologue overlaps the previous kernel's tail
        cudaLaunchConfig_t cfg{};
        cfg.gridDim = dim3((unsigned)R.nparts);
        cfg.blockDim = dim3(wide_threads<MODE>());
        cfg.dynamicSmemBytes = smem;
        cfg.stream = s;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        at[0].val.programmaticStreamSerializationAllowed = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        const cudaError_t le = cudaLaunchKernelEx(&cfg, k_sector_run_wide<MODE, T, DSW>, static_cast<V*>(psi),
                                                  static_cast<V*>(lam), R, parts, blks, partial, pmax, cm,
                                                  static_cast<V*>(log), strs, map, DSW && dss);
        if (le != cudaSuccess) return le;
      }
    }
    if constexpr (!DSW)
      if (!wide)
        k_sector_run<MODE, T><<<R.nparts, kRunThreads, smem, s>>>(
            static_cast<V*>(psi), static_cast<V*>(lam), R, parts, blks, partial, pmax, cm, static_cast<V*>(log),
            strs, (MODE == 0 || MODE == 3) ? map : nullptr, false);
    count_launch();
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t launch_sector_runs(void* psi, void* lam, qf_dtype dt, bool adj, bool realst, const RunInfo* runs,
                               int nruns, const RunPart* parts, const RunBlk* blks, int nblk, double* partial,
                               int pmax, double* out, const SecCompact& cm, void* log, const uint16_t* strs,
                               const uint32_t* map, bool ds, bool dss, cudaStream_t s) {
  if (nblk <= 0 || nruns <= 0) return cudaSuccess;
  if (!cm.ra || (log && !realst)) return cudaErrorInvalidValue;
  const bool dsw = dt == QF_C128 && ds && map && (!adj || (realst && log));
  if (dss && !dsw) return cudaErrorInvalidValue;  // the double-single layout needs the double-single sweeps
  const int prof_slot_ = prof_pre(adj ? QF_K_ADJ_SPARSE : QF_K_SPARSE, s);
  const int mode = !adj ? 0 : !realst ? 2 : log ? 3 : 1;
  cudaError_t e;
  if (dsw)
    e = mode == 0 ? runs_t<0, double, true>(psi, lam, runs, nruns, parts, blks, partial, pmax, cm, log, strs, map, dss, s)
                  : runs_t<3, double, true>(psi, lam, runs, nruns, parts, blks, partial, pmax, cm, log, strs, map, dss, s);
  else if (dt == QF_C128)
    e = mode == 0 ? runs_t<0, double>(psi, lam, runs, nruns, parts, blks, partial, pmax, cm, log, strs, map, dss, s)
      : mode == 1 ? runs_t<1, double>(psi, lam, runs, nruns, parts, blks, partial, pmax, cm, log, strs, map, dss, s)
      : mode == 2 ? runs_t<2, double>(psi, lam, runs, nruns, parts, blks, partial, pmax, cm, log, strs, map, dss, s)
                  : runs_t<3, double>(psi, lam, runs, nruns, parts, blks, partial, pmax, cm, log, strs, map, dss, s);
  else
    e = mode == 0 ? runs_t<0, float>(psi, lam, runs, nruns, parts, blks, partial, pmax, cm, log, strs, map, dss, s)
      : mode == 1 ? runs_t<1, float>(psi, lam, runs, nruns, parts, blks, partial, pmax, cm, log, strs, map, dss, s)
      : mode == 2 ? runs_t<2, float>(psi, lam, runs, nruns, parts, blks, partial, pmax, cm, log, strs, map, dss, s)
                  : runs_t<3, float>(psi, lam, runs, nruns, parts, blks, partial, pmax, cm, log, strs, map, dss, s);
  if (e == cudaSuccess && adj) {
    k_sector_reduce_parts<<<(nblk + 7) / 8, 256, 0, s>>>(partial, pmax, blks, nblk, out);
    e = cudaGetLastError();
    count_launch();
  }
  prof_post(prof_slot_, s);
  return e;
}

cudaError_t launch_run_itemmaps(const RunInfo* runs, int nruns, const RunPart* parts, const RunBlk* blks,
                                const SecCompact& cm, const uint16_t* strs, uint32_t* map, cudaStream_t s) {
  if (!cm.ra || !map) return cudaErrorInvalidValue;
  for (int r = 0; r < nruns; ++r) {
    if (runs[r].nparts <= 0) continue;
    if (runs[r].maxsize > kMapMaxPart) return cudaErrorInvalidValue;
    k_run_itemmap<<<runs[r].nparts, kRunThreads, 0, s>>>(runs[r], parts, blks, cm, strs, map);
    count_launch();
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t launch_sector_overlaps(void* psi, qf_dtype dt, const RunInfo* runs, int nruns, const RunPart* parts,
                                  const RunBlk* blks, int nblk, double* partial, int pmax, double* out,
                                  const SecCompact& cm, const uint16_t* strs, cudaStream_t s) {
  if (nblk <= 0 || nruns <= 0) return cudaSuccess;
  if (!cm.ra) return cudaErrorInvalidValue;
  const int prof_slot_ = prof_pre(QF_K_ADJ_SPARSE, s);
  cudaError_t e = (dt == QF_C128)
                      ? runs_t<4, double>(psi, psi, runs, nruns, parts, blks, partial, pmax, cm, nullptr, strs, nullptr, false, s)
                      : runs_t<4, float>(psi, psi, runs, nruns, parts, blks, partial, pmax, cm, nullptr, strs, nullptr, false, s);
  if (e == cudaSuccess) {
    k_sector_reduce_parts<<<(nblk + 7) / 8, 256, 0, s>>>(partial, pmax, blks, nblk, out);
    e = cudaGetLastError();
    count_launch();
  }
  prof_post(prof_slot_, s);
  return e;
}

// Grid of the sector H|psi>: every CTA the SMs hold at once (grid-stride loop
// over members), at most max_blocks (the reduction's partial slots).
template <typename K>
static unsigned hpsi_grid(K kernel, uint64_t items, int max_blocks) {
  static const int resident = [&] {  // one per kernel instantiation, initialised once
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, 256, 0);
    return std::max(1, sms) * std::max(1, per_sm);
  }();
  const uint64_t want = (items + 255) / 256;
  return (unsigned)std::max<uint64_t>(1, std::min<uint64_t>(want, (uint64_t)std::min(resident, max_blocks)));
}

template <typename T, bool REALST, bool LAMY, bool COMPACT>
static void hpsi_t(const void* psi, void* lam, bool narrow, int max_blocks, const SecSpace& sp, const SecRank& rk,
                   const SecGroup* large, int nlarge, const ExpChunk* chunks, double* partials,
                   unsigned* counter, double* out, const SecCompact& cm, cudaStream_t s) {
  using V = typename SCx<T>::V;
  const V* p = static_cast<const V*>(psi);
  V* l = static_cast<V*>(lam);
  const uint64_t items = (uint64_t)sp.cnt_e * sp.cnt_o;
  if (narrow) {
    const auto k = k_sector_hpsi<T, REALST, true, LAMY, COMPACT>;
    k<<<hpsi_grid(k, items, max_blocks), 256, 0, s>>>(p, l, sp, rk, large, nlarge, chunks, partials, counter,
                                                      out, cm);
  } else {
    const auto k = k_sector_hpsi<T, REALST, false, LAMY, COMPACT>;
    k<<<hpsi_grid(k, items, max_blocks), 256, 0, s>>>(p, l, sp, rk, large, nlarge, chunks, partials, counter,
                                                      out, cm);
  }
}

template <typename T>
static cudaError_t hpsi_dispatch(const void* psi, void* lam, bool realst, bool narrow, int g,
                                 const SecSpace& sp, const SecRank& rk,
                                 const SecGroup* large, int nlarge, const ExpChunk* chunks, double* partials,
                                 unsigned* counter, double* out, const SecCompact& cm, cudaStream_t s) {
  const bool lamy = realst && lam == psi;  // packed: lambda into psi's imaginary slots
  if (!cm.ra) {  // full layout (expectation values): no packed lambda
    if (lamy) return cudaErrorInvalidValue;
    if (realst)
      hpsi_t<T, true, false, false>(psi, lam, narrow, g, sp, rk, large, nlarge, chunks, partials, counter, out,
                                    cm, s);
    else
      hpsi_t<T, false, false, false>(psi, lam, narrow, g, sp, rk, large, nlarge, chunks, partials, counter,
                                     out, cm, s);
    return cudaGetLastError();
  }
  // compact layout (energy and gradient): a real lambda is always packed
  if (realst != lamy) return cudaErrorInvalidValue;
  if (lamy)
    hpsi_t<T, true, true, true>(psi, lam, narrow, g, sp, rk, large, nlarge, chunks, partials, counter, out, cm,
                                s);
  else
    hpsi_t<T, false, false, true>(psi, lam, narrow, g, sp, rk, large, nlarge, chunks, partials, counter, out,
                                  cm, s);
  return cudaGetLastError();
}

cudaError_t launch_sector_hpsi_direct(void* cpsi, qf_dtype dt, const SecSpace& sp, const SecDirect& d,
                                      const SecCompact& cm, double* partials, unsigned* counter, double* out,
                                      int nblocks, float2* split, double* psid, bool dss, cudaStream_t s) {
  if (d.n > 32 || d.ne != sp.ne || d.no != sp.no || sp.ne > 16) return cudaErrorInvalidValue;
  if (dss && (dt != QF_C128 || !split || !psid)) return cudaErrorInvalidValue;
  // the beta-single lists: ko (no - ko) entries per thread (at most 64 at 32 qubits);
  // partner ranks must fit 14 bits
  if (sp.cnt_o > (1u << 14)) return cudaErrorInvalidValue;
  const size_t smem = (size_t)std::max(1, sp.ko * (sp.no - sp.ko)) * 256 * sizeof(uint32_t);
  const int prof_slot_ = prof_pre(QF_K_HPSI, s);
  const uint64_t items = (uint64_t)sp.cnt_e * sp.cnt_o;
  auto grid = [&](auto kernel) {  // every CTA the SMs hold at this shared-memory size
    static std::once_flag once;
    std::call_once(once, [&] {
      cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 64 * 256 * (int)sizeof(uint32_t));
    });
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, 256, smem);
    const uint64_t want = (items + 255) / 256;
    const uint64_t res = (uint64_t)std::max(1, sms) * (uint64_t)std::max(1, per_sm);
    return (unsigned)std::max<uint64_t>(1, std::min<uint64_t>(want, std::min<uint64_t>(res, (uint64_t)nblocks)));
  };
  if (dt == QF_C128 && split) {
    k_split_real<<<(unsigned)std::min<uint64_t>((items + 255) / 256, 4096), 256, 0, s>>>(
        static_cast<const double*>(cpsi), split, psid, items, dss);
    count_launch();
    const auto k = k_sector_hpsi_direct<double, true>;
    k<<<grid(k), 256, smem, s>>>(static_cast<double*>(cpsi), d, sp.cnt_e, sp.cnt_o, sp.ke, sp.ko, cm.ra, cm.rb,
                                 partials, counter, out, split, psid, dss);
  } else if (dt == QF_C128) {
    const auto k = k_sector_hpsi_direct<double, false>;
    k<<<grid(k), 256, smem, s>>>(static_cast<double*>(cpsi), d, sp.cnt_e, sp.cnt_o, sp.ke, sp.ko, cm.ra, cm.rb,
                                 partials, counter, out, nullptr, nullptr, false);
  } else {
    const auto k = k_sector_hpsi_direct<float, false>;
    k<<<grid(k), 256, smem, s>>>(static_cast<float*>(cpsi), d, sp.cnt_e, sp.cnt_o, sp.ke, sp.ko, cm.ra, cm.rb,
                                 partials, counter, out, nullptr, nullptr, false);
  }
  const cudaError_t e = cudaGetLastError();
  prof_post(prof_slot_, s);
  count_launch();
  return e;
}

cudaError_t launch_sector_hpsi(const void* psi, void* lam, qf_dtype dt, bool realst, const SecSpace& sp,
                               const SecRank& rk, const SecGroup* large, int nlarge,
                               const ExpChunk* chunks, double* partials, unsigned* counter, double* out,
                               int nblocks, const SecCompact& cm, cudaStream_t s) {
  const int prof_slot_ = prof_pre(QF_K_HPSI, s);
  const int g = nblocks;  // partial slots available: the grid's upper bound
  const bool narrow = sp.ne + sp.no <= 32;
  const cudaError_t e =
      (dt == QF_C128)
          ? hpsi_dispatch<double>(psi, lam, realst, narrow, g, sp, rk, large, nlarge, chunks, partials, counter,
                                  out, cm, s)
          : hpsi_dispatch<float>(psi, lam, realst, narrow, g, sp, rk, large, nlarge, chunks, partials, counter,
                                 out, cm, s);
  prof_post(prof_slot_, s);
  count_launch();
  return e;
}

size_t small_eval_smem(qf_dtype dt, uint32_t members, int ko, int no) {
  const size_t real = dt == QF_C128 ? sizeof(double) : sizeof(float);
  const size_t b = align16(2 * (size_t)members * real) +
                   (size_t)std::max(1, ko * (no - ko)) * kSmallThreads * sizeof(uint32_t);
  return b <= 200u * 1024u ? b : 0;
}

cudaError_t launch_small_eval(const SmallEval& a, qf_dtype dt, int n_req, cudaStream_t s) {
  if (n_req <= 0 || a.nblk < 0) return cudaSuccess;
  const size_t smem = small_eval_smem(dt, a.cnt_e * a.cnt_o, a.ko, a.d.no);
  if (smem == 0 || a.d.n > 32 || a.cnt_o > (1u << 14)) return cudaErrorInvalidValue;
  const auto k = dt == QF_C128 ? k_small_eval<double> : k_small_eval<float>;
  static std::once_flag once_d, once_f;  // allow the opt-in shared memory size, once per process
  static cudaError_t attr_d = cudaSuccess, attr_f = cudaSuccess;
  if (dt == QF_C128)
    std::call_once(once_d, [&] {
      attr_d = cudaFuncSetAttribute(k_small_eval<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    });
  else
    std::call_once(once_f, [&] {
      attr_f = cudaFuncSetAttribute(k_small_eval<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    });
  const cudaError_t attr = dt == QF_C128 ? attr_d : attr_f;
  if (attr != cudaSuccess) return attr;
  const int prof_slot_ = prof_pre(QF_K_SPARSE, s);
  k<<<n_req, kSmallThreads, smem, s>>>(a);
  count_launch();
  const cudaError_t e = cudaGetLastError();
  prof_post(prof_slot_, s);
  return e;
}

}  // namespace qf
