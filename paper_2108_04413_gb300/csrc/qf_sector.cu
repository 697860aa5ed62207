// Sector-restricted kernels.
//
// A state built from a basis determinant by particle-number- and S_z-
// conserving blocks (every spin-conserving dUCC excitation, Eq. 19) has nonzero
// amplitudes only on determinants with the reference's number of occupied even
// qubits (alpha spin orbitals) and odd qubits (beta): C(n/2, N_a) * C(n/2, N_b)
// of the 2^n basis states, 5 % at 24 qubits.  Restricting the state to that
// sector is the speed-up the paper's conclusion proposes for larger systems.
// The state keeps its full 2^n layout here; these kernels simply enumerate the
// sector members by combinatorial unranking and never touch the (exactly zero)
// amplitudes outside it.
//
// * k_sector_sweep: every excitation block of a circuit in one persistent
//   cooperative launch, with a grid barrier between consecutive blocks; for the
//   reverse sweep it also records each block's gradient overlap per CTA.
// * k_sector_hpsi: lambda = H psi on the sector members only (the only part
//   that enters <psi|lambda>, the gradient overlaps and the reverse sweep, since
//   psi and every block stay in the sector), with <psi|lambda> and <psi|psi>.
//
// Grid barriers spin with an iteration limit; on timeout a block raises the
// error flag and every block leaves at its next barrier.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "qf_internal.h"

namespace qf {
namespace {

constexpr int kBinom = 18;  // C(m, k) for m, k < 18 (up to 34 qubits: 17 per parity)

__device__ __forceinline__ unsigned par64s(uint64_t v) { return (unsigned)__popcll(v) & 1u; }

__device__ void fill_binom(uint32_t (*C)[kBinom]) {
  for (int i = threadIdx.x; i < kBinom * kBinom; i += blockDim.x) {
    const int m = i / kBinom, k = i % kBinom;
    // C(m, k) by the multiplicative formula (exact in 64-bit for m < 18)
    uint64_t c = (k > m) ? 0 : 1;
    for (int j = 1; j <= k && k <= m; ++j) c = c * (uint64_t)(m - k + j) / (uint64_t)j;
    C[m][k] = (uint32_t)c;
  }
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

constexpr long long kSpinLimit = 1ll << 26;

// Grid-wide barrier with a bounded wait.  bar[0] = arrivals, bar[1] = generation,
// bar[2] = error flag.  Returns false when the grid must stop (error raised).
__device__ bool grid_barrier(unsigned* bar) {
  __shared__ int stop;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned* vgen = bar + 1;
    volatile unsigned* verr = bar + 2;
    const unsigned gen = *vgen;
    __threadfence();
    const unsigned arrived = atomicAdd(bar, 1u);
    if (arrived == gridDim.x - 1) {
      atomicExch(bar, 0u);
      __threadfence();
      atomicAdd(bar + 1, 1u);
    } else {
      long long it = 0;
      while (*vgen == gen && *verr == 0u) {
        if (++it > kSpinLimit) {
          atomicExch(bar + 2, 1u);
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
    stop = (*verr != 0u);
  }
  __syncthreads();
  return !stop;
}

template <typename T> struct SCx;
template <> struct SCx<double> { using V = double2; };
template <> struct SCx<float> { using V = float2; };

// One excitation block of a sector sweep (forward or reverse): the real 2x2
// composite minus identity per sign class and, for the reverse sweep, the real
// matrix Qi with Q = i Qi.
template <bool ADJ, bool REALST, typename T>
__device__ void sector_block(typename SCx<T>::V* psi, typename SCx<T>::V* lam, const SecBlk& B,
                             const uint32_t (*C)[kBinom], double* acc_out) {
  using V = typename SCx<T>::V;
  const uint64_t items = (uint64_t)B.cnt_e * (uint64_t)B.cnt_o;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  double acc = 0.0;
  T* pr = reinterpret_cast<T*>(psi);
  T* lr = reinterpret_cast<T*>(lam);
  for (uint64_t it = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; it < items; it += stride) {
    const uint32_t ie = (uint32_t)(it / B.cnt_o), io = (uint32_t)(it % B.cnt_o);
    const uint64_t base = unrank(ie, B.epos, B.ne, B.ke, C) | unrank(io, B.opos, B.no, B.ko, C);
    unsigned cls = 0;
    if (B.nzc > 0) cls = par64s(B.zc[0] & base);
    if (B.nzc > 1) cls |= par64s(B.zc[1] & base) << 1;
    const uint64_t i0 = base | B.pat[0], i1 = base | B.pat[1];
    const T a00 = (T)B.m[cls][0][0], a01 = (T)B.m[cls][0][1], a10 = (T)B.m[cls][1][0], a11 = (T)B.m[cls][1][1];
    // L2-coherent accesses: other SMs wrote these amplitudes before the last grid barrier
    if (REALST) {
      const T v0 = __ldcg(pr + 2 * i0), v1 = __ldcg(pr + 2 * i1);
      if (ADJ) {
        const T w0 = __ldcg(lr + 2 * i0), w1 = __ldcg(lr + 2 * i1);
        // Im <lam|Q|psi> = Re <lam|Qi|psi> for real Qi
        acc = fma((double)w0, fma(B.q[cls][0][0], (double)v0, B.q[cls][0][1] * (double)v1), acc);
        acc = fma((double)w1, fma(B.q[cls][1][0], (double)v0, B.q[cls][1][1] * (double)v1), acc);
        __stcg(lr + 2 * i0, fma(a00, w0, fma(a01, w1, w0)));
        __stcg(lr + 2 * i1, fma(a10, w0, fma(a11, w1, w1)));
      }
      __stcg(pr + 2 * i0, fma(a00, v0, fma(a01, v1, v0)));
      __stcg(pr + 2 * i1, fma(a10, v0, fma(a11, v1, v1)));
    } else {
      const V v0 = __ldcg(psi + i0), v1 = __ldcg(psi + i1);
      if (ADJ) {
        const V w0 = __ldcg(lam + i0), w1 = __ldcg(lam + i1);
        const double q00 = B.q[cls][0][0], q01 = B.q[cls][0][1], q10 = B.q[cls][1][0], q11 = B.q[cls][1][1];
        acc += (double)w0.x * (q00 * v0.x + q01 * v1.x) + (double)w0.y * (q00 * v0.y + q01 * v1.y);
        acc += (double)w1.x * (q10 * v0.x + q11 * v1.x) + (double)w1.y * (q10 * v0.y + q11 * v1.y);
        V o0, o1;
        o0.x = fma(a00, w0.x, fma(a01, w1.x, w0.x));
        o0.y = fma(a00, w0.y, fma(a01, w1.y, w0.y));
        o1.x = fma(a10, w0.x, fma(a11, w1.x, w1.x));
        o1.y = fma(a10, w0.y, fma(a11, w1.y, w1.y));
        __stcg(lam + i0, o0);
        __stcg(lam + i1, o1);
      }
      V o0, o1;
      o0.x = fma(a00, v0.x, fma(a01, v1.x, v0.x));
      o0.y = fma(a00, v0.y, fma(a01, v1.y, v0.y));
      o1.x = fma(a10, v0.x, fma(a11, v1.x, v1.x));
      o1.y = fma(a10, v0.y, fma(a11, v1.y, v1.y));
      __stcg(psi + i0, o0);
      __stcg(psi + i1, o1);
    }
  }
  if (ADJ) *acc_out = acc;
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

// Persistent sweep over blocks [0, nblk) (forward: in order; reverse: from the
// last).  Reverse: partial[b * gridDim.x + blockIdx.x] receives block b's
// overlap summed over this CTA.
template <bool ADJ, bool REALST, typename T>
__global__ void __launch_bounds__(256) k_sector_sweep(typename SCx<T>::V* psi, typename SCx<T>::V* lam,
                                                      const SecBlk* __restrict__ blks, int nblk, unsigned* bar,
                                                      double* partial) {
  __shared__ uint32_t C[kBinom][kBinom];
  __shared__ SecBlk sb;  // the current block's description, read by every thread
  fill_binom(C);
  for (int s = 0; s < nblk; ++s) {
    const int b = ADJ ? (nblk - 1 - s) : s;
    __syncthreads();
    {
      const uint32_t* src = reinterpret_cast<const uint32_t*>(blks + b);
      uint32_t* dst = reinterpret_cast<uint32_t*>(&sb);
      for (int i = threadIdx.x; i < (int)(sizeof(SecBlk) / 4); i += blockDim.x) dst[i] = __ldcg(src + i);
    }
    __syncthreads();
    double acc = 0.0;
    sector_block<ADJ, REALST, T>(psi, lam, sb, C, &acc);
    if (ADJ) {
      acc = block_sum_s(acc);
      if (threadIdx.x == 0) partial[(size_t)b * gridDim.x + blockIdx.x] = acc;
    }
    if (s + 1 < nblk && !grid_barrier(bar)) return;
  }
}

// out[b] = sum over CTAs of partial[b * ncta + cta], in CTA order.
__global__ void k_sector_reduce_rows(const double* __restrict__ partial, int ncta, int nblk, double* out) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nblk) return;
  double s = 0.0;
  for (int c = 0; c < ncta; ++c) s += partial[(size_t)b * ncta + c];
  out[b] = s;
}

// lambda = H psi on the sector members; out[0] = <psi|lambda>, out[1] = <psi|psi>
// (block partials reduced by the last block, in order).
template <typename T, bool REALST>
__global__ void __launch_bounds__(256) k_sector_hpsi(const typename SCx<T>::V* __restrict__ psi,
                                                     typename SCx<T>::V* __restrict__ lam, SecSpace sp,
                                                     const SecGroup* __restrict__ groups, int ngroups,
                                                     const ExpChunk* __restrict__ chunks, double* partials,
                                                     unsigned* counter, double* out) {
  using V = typename SCx<T>::V;
  __shared__ uint32_t C[kBinom][kBinom];
  constexpr int kBatch = 512;
  __shared__ SecGroup sg[kBatch];
  __shared__ SecSpace ssp;
  fill_binom(C);
  if (threadIdx.x == 0) ssp = sp;
  __syncthreads();
  const uint64_t items = (uint64_t)sp.cnt_e * (uint64_t)sp.cnt_o;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  const uint64_t EVEN = 0x5555555555555555ull, ODD = 0xAAAAAAAAAAAAAAAAull;
  double acc_e = 0.0, acc_n = 0.0;
  // every thread runs the same number of item rounds so the group batches stay in step
  const uint64_t rounds = (items + stride - 1) / stride;
  for (uint64_t rd = 0; rd < rounds; ++rd) {
    const uint64_t it = rd * stride + blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    const bool live = it < items;
    uint64_t c = 0;
    if (live) {
      const uint32_t ie = (uint32_t)(it / ssp.cnt_o), io = (uint32_t)(it % ssp.cnt_o);
      c = unrank(ie, ssp.epos, ssp.ne, ssp.ke, C) | unrank(io, ssp.opos, ssp.no, ssp.ko, C);
    }
    double lx = 0.0, ly = 0.0;
    for (int g0 = 0; g0 < ngroups; g0 += kBatch) {
      const int nb = min(kBatch, ngroups - g0);
      __syncthreads();
      for (int i = threadIdx.x; i < nb; i += blockDim.x) sg[i] = groups[g0 + i];
      __syncthreads();
      if (!live) continue;
      for (int i = 0; i < nb; ++i) {
        const SecGroup G = sg[i];
        // the partner c ^ x is in the sector iff x flips as many occupied as empty
        // even (and odd) qubits of c
        if (2 * __popcll(c & G.x & EVEN) != G.xe || 2 * __popcll(c & G.x & ODD) != G.xo) continue;
        const uint64_t b = c ^ G.x;
        double dx = 0.0, dy = 0.0;
        for (int k = 0; k < G.nchunk; ++k) {
          const ExpChunk* W = chunks + G.chunk0 + k;
          unsigned idx = 0;
#pragma unroll
          for (int t = 0; t < kChunkTerms; ++t) idx |= par64s(W->z[t] & b) << t;
          const double2 d = W->tab[idx];
          dx += d.x;
          dy += d.y;
        }
        const V v = psi[b];
        lx = fma(dx, (double)v.x, lx);
        if (!REALST) {
          lx = fma(-dy, (double)v.y, lx);
          ly = fma(dx, (double)v.y, fma(dy, (double)v.x, ly));
        }
      }
    }
    if (live) {
      const V u = psi[c];
      acc_e = fma((double)u.x, lx, fma((double)u.y, ly, acc_e));
      acc_n = fma((double)u.x, (double)u.x, fma((double)u.y, (double)u.y, acc_n));
      if (lam) {
        V w;
        w.x = (T)lx;
        w.y = (T)ly;
        lam[c] = w;
      }
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

}  // namespace

// Largest grid the cooperative sweep can use (every CTA resident at once).
template <bool ADJ, bool REALST, typename T>
static int sweep_grid() {
  int per_sm = 0, dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_sector_sweep<ADJ, REALST, T>, 256, 0);
  return std::max(1, std::min(per_sm, 4)) * std::max(1, sms);
}

template <bool ADJ, bool REALST, typename T>
static cudaError_t sweep_t(void* psi, void* lam, const SecBlk* blks, int nblk, unsigned* bar, double* partial,
                           int grid, cudaStream_t s) {
  using V = typename SCx<T>::V;
  V* p = static_cast<V*>(psi);
  V* l = static_cast<V*>(lam);
  void* args[] = {&p, &l, &blks, &nblk, &bar, &partial};
  return cudaLaunchCooperativeKernel((const void*)k_sector_sweep<ADJ, REALST, T>, dim3(grid), dim3(256), args, 0, s);
}

int sector_sweep_grid(qf_dtype dt, bool adj, bool realst) {
  if (dt == QF_C128) {
    if (adj) return realst ? sweep_grid<true, true, double>() : sweep_grid<true, false, double>();
    return realst ? sweep_grid<false, true, double>() : sweep_grid<false, false, double>();
  }
  if (adj) return realst ? sweep_grid<true, true, float>() : sweep_grid<true, false, float>();
  return realst ? sweep_grid<false, true, float>() : sweep_grid<false, false, float>();
}

cudaError_t launch_sector_sweep(void* psi, void* lam, qf_dtype dt, bool adj, bool realst, const SecBlk* blks,
                                int nblk, unsigned* bar, double* partial, double* out, int grid, cudaStream_t s) {
  if (nblk <= 0) return cudaSuccess;
  const int prof_slot_ = prof_pre(adj ? QF_K_ADJ_SPARSE : QF_K_SPARSE, s);
  cudaError_t e = cudaMemsetAsync(bar, 0, 3 * sizeof(unsigned), s);
  if (e == cudaSuccess) {
    if (dt == QF_C128) {
      if (adj)
        e = realst ? sweep_t<true, true, double>(psi, lam, blks, nblk, bar, partial, grid, s)
                   : sweep_t<true, false, double>(psi, lam, blks, nblk, bar, partial, grid, s);
      else
        e = realst ? sweep_t<false, true, double>(psi, lam, blks, nblk, bar, partial, grid, s)
                   : sweep_t<false, false, double>(psi, lam, blks, nblk, bar, partial, grid, s);
    } else {
      if (adj)
        e = realst ? sweep_t<true, true, float>(psi, lam, blks, nblk, bar, partial, grid, s)
                   : sweep_t<true, false, float>(psi, lam, blks, nblk, bar, partial, grid, s);
      else
        e = realst ? sweep_t<false, true, float>(psi, lam, blks, nblk, bar, partial, grid, s)
                   : sweep_t<false, false, float>(psi, lam, blks, nblk, bar, partial, grid, s);
    }
  }
  count_launch();
  if (e == cudaSuccess && adj) {
    k_sector_reduce_rows<<<(nblk + 255) / 256, 256, 0, s>>>(partial, grid, nblk, out);
    e = cudaGetLastError();
    count_launch();
  }
  prof_post(prof_slot_, s);
  return e;
}

cudaError_t launch_sector_hpsi(const void* psi, void* lam, qf_dtype dt, bool realst, const SecSpace& sp,
                               const SecGroup* groups, int ngroups, const ExpChunk* chunks, double* partials,
                               unsigned* counter, double* out, int nblocks, cudaStream_t s) {
  const int prof_slot_ = prof_pre(QF_K_HPSI, s);
  const uint64_t items = (uint64_t)sp.cnt_e * sp.cnt_o;
  const unsigned g = (unsigned)std::max<uint64_t>(1, std::min<uint64_t>((items + 255) / 256, (uint64_t)nblocks));
  if (dt == QF_C128) {
    if (realst)
      k_sector_hpsi<double, true><<<g, 256, 0, s>>>(static_cast<const double2*>(psi), static_cast<double2*>(lam), sp,
                                                    groups, ngroups, chunks, partials, counter, out);
    else
      k_sector_hpsi<double, false><<<g, 256, 0, s>>>(static_cast<const double2*>(psi), static_cast<double2*>(lam),
                                                     sp, groups, ngroups, chunks, partials, counter, out);
  } else {
    if (realst)
      k_sector_hpsi<float, true><<<g, 256, 0, s>>>(static_cast<const float2*>(psi), static_cast<float2*>(lam), sp,
                                                   groups, ngroups, chunks, partials, counter, out);
    else
      k_sector_hpsi<float, false><<<g, 256, 0, s>>>(static_cast<const float2*>(psi), static_cast<float2*>(lam), sp,
                                                    groups, ngroups, chunks, partials, counter, out);
  }
  prof_post(prof_slot_, s);
  count_launch();
  return cudaGetLastError();
}

}  // namespace qf
