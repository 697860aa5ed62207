// CUDA kernels of libqf for GB300 (sm_103a).
//
// Every kernel streams the 2^n-amplitude state vector (interleaved complex,
// double2 for complex128, float2 for complex64).  The rotation kernels apply
// exp(-i theta P) (Eq. 9, with the factor -i theta of Eq. 11) as a pair swap
// b <-> b xor x with the phase i^{popc(x&z)} (-1)^{popc(z&b)} of the Pauli
// string (Eq. 10); the expectation kernels evaluate exact operator averaging
// (Eq. 18) with the terms grouped by X mask.  Reductions are FP64 for both
// state precisions and deterministic (fixed-order second stage).
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "qf_internal.h"

namespace qf {

namespace {

template <typename T> struct Cx;
template <> struct Cx<double> { using V = double2; };
template <> struct Cx<float> { using V = float2; };

__device__ __forceinline__ double flip(double v, unsigned neg) {
  return __longlong_as_double(__double_as_longlong(v) ^ ((unsigned long long)(neg & 1u) << 63));
}
__device__ __forceinline__ float flip(float v, unsigned neg) {
  return __int_as_float(__float_as_int(v) ^ (int)((neg & 1u) << 31));
}

// i^k * v for k in 0..3, done with component swaps and sign-bit flips only.
template <typename V>
__device__ __forceinline__ V qturn(V v, unsigned k) {
  V o;
  o.x = flip((k & 1u) ? v.y : v.x, (k ^ (k >> 1)) & 1u);
  o.y = flip((k & 1u) ? v.x : v.y, (k >> 1) & 1u);
  return o;
}

// The form is a compile-time parameter: with a runtime form the compiler
// evaluates every branch, tripling the FP64 work of the one-FMA forms.
template <int F, typename T, typename V>
__device__ __forceinline__ V comb(V u, V w, T A, T B) {
  V o;
  if (F == FORM_A1) {
    o.x = fma(B, w.x, u.x);
    o.y = fma(B, w.y, u.y);
  } else if (F == FORM_B1) {
    o.x = fma(A, u.x, w.x);
    o.y = fma(A, u.y, w.y);
  } else {
    o.x = fma(B, w.x, A * u.x);
    o.y = fma(B, w.y, A * u.y);
  }
  return o;
}

__device__ __forceinline__ uint64_t ins0(uint64_t p, int h) {
  return ((p >> h) << (h + 1)) | (p & ((1ull << h) - 1ull));
}

__device__ __forceinline__ unsigned par64(uint64_t v) { return (unsigned)__popcll(v) & 1u; }

// ---------------------------------------------------------------------------
// deterministic block + grid reduction (the last block to finish sums the
// per-block partials in index order)

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

__device__ double block_sum(double v) {
  __shared__ double red[32];
  __syncthreads();
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) red[wid] = v;
  __syncthreads();
  const int nw = (blockDim.x + 31) >> 5;
  v = (threadIdx.x < nw) ? red[threadIdx.x] : 0.0;
  if (wid == 0) v = warp_sum(v);
  return v;  // valid in thread 0
}

__device__ void grid_finish(double v, double* partials, unsigned* counter, double* out) {
  __shared__ bool last;
  double bs = block_sum(v);
  if (threadIdx.x == 0) {
    partials[blockIdx.x] = bs;
    __threadfence();
    unsigned t = atomicAdd(counter, 1u);
    last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (last) {
    __threadfence();
    double s = 0.0;
    for (unsigned i = threadIdx.x; i < gridDim.x; i += blockDim.x) s += __ldcg(partials + i);
    s = block_sum(s);
    if (threadIdx.x == 0) {
      *out = s;
      *counter = 0u;
    }
  }
}

// Two sums at once (out[0], out[1]); partials holds 2 * gridDim.x doubles.
__device__ void grid_finish2(double v0, double v1, double* partials, unsigned* counter, double* out) {
  __shared__ bool last2;
  const double b0 = block_sum(v0);
  const double b1 = block_sum(v1);
  if (threadIdx.x == 0) {
    partials[2 * blockIdx.x] = b0;
    partials[2 * blockIdx.x + 1] = b1;
    __threadfence();
    unsigned t = atomicAdd(counter, 1u);
    last2 = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (last2) {
    __threadfence();
    double s0 = 0.0, s1 = 0.0;
    for (unsigned i = threadIdx.x; i < gridDim.x; i += blockDim.x) {
      s0 += __ldcg(partials + 2 * i);
      s1 += __ldcg(partials + 2 * i + 1);
    }
    s0 = block_sum(s0);
    s1 = block_sum(s1);
    if (threadIdx.x == 0) {
      out[0] = s0;
      out[1] = s1;
      *counter = 0u;
    }
  }
}

// ---------------------------------------------------------------------------
// state preparation

template <typename V>
__global__ void k_zero_and_set(V* psi, uint64_t N, uint64_t det) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < N; i += stride) {
    V v;
    v.x = (i == det) ? 1 : 0;
    v.y = 0;
    psi[i] = v;
  }
}

// out[2k], out[2k + 1] = the amplitude at idx[k] (0 where idx[k] < 0); packed:
// the real value stored in the imaginary slot, imaginary part 0.
// The same for a packed double-single state: (re hi, re lo, packed hi, packed lo).
__global__ void k_gather_ds(const float4* __restrict__ src, const int64_t* __restrict__ idx, int count,
                            double* __restrict__ out) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= count) return;
  const int64_t i = idx[k];
  double re = 0.0;
  if (i >= 0) {
    const float4 v = src[i];
    re = (double)v.z + (double)v.w;
  }
  out[2 * k] = re;
  out[2 * k + 1] = 0.0;
}

template <typename V>
__global__ void k_gather(const V* __restrict__ src, const int64_t* __restrict__ idx, int count, int packed,
                         double* __restrict__ out) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= count) return;
  const int64_t i = idx[k];
  double re = 0.0, im = 0.0;
  if (i >= 0) {
    const V v = src[i];
    if (packed) {
      re = (double)v.y;
    } else {
      re = (double)v.x;
      im = (double)v.y;
    }
  }
  out[2 * k] = re;
  out[2 * k + 1] = im;
}

template <typename T>
__global__ void k_scale(typename Cx<T>::V* psi, uint64_t N, T s) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < N; i += stride) {
    auto v = psi[i];
    v.x *= s;
    v.y *= s;
    psi[i] = v;
  }
}

// ---------------------------------------------------------------------------
// unfused rotation: one read + one write sweep of the state
//
// For the pair (b, b' = b xor x) with b's pivot bit h clear and par = popc(z&b) mod 2:
//   out[b]  = A u + B i^{3+3y+2par} v,     out[b'] = A v + B i^{3+y+2par} u,
// which is c u - i s (P psi)[b] etc. with A = c, B = s (up to the kept scale).
// Each thread takes the two pairs (b, b|1) so the partner amplitudes also form
// an aligned 2-vector (needs h >= 1).

template <typename T, int F>
__global__ void __launch_bounds__(256) k_rot_pair2(typename Cx<T>::V* __restrict__ psi, uint64_t nquads, uint64_t x,
                                                   uint64_t z, int h, int y, T A, T B) {
  using V = typename Cx<T>::V;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  const unsigned z0 = (unsigned)(z & 1ull);
  for (uint64_t q = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; q < nquads; q += stride) {
    const uint64_t b0 = ins0(q << 1, h);  // even, pivot clear
    const uint64_t b1 = b0 | 1ull;
    const uint64_t c0 = b0 ^ x, c1 = b1 ^ x;
    const V u0 = psi[b0], u1 = psi[b1];
    const V v0 = psi[c0], v1 = psi[c1];
    const unsigned p0 = par64(z & b0), p1 = p0 ^ z0;
    psi[b0] = comb<F, T, V>(u0, qturn(v0, (3u + 3u * y + 2u * p0) & 3u), A, B);
    psi[b1] = comb<F, T, V>(u1, qturn(v1, (3u + 3u * y + 2u * p1) & 3u), A, B);
    psi[c0] = comb<F, T, V>(v0, qturn(u0, (3u + y + 2u * p0) & 3u), A, B);
    psi[c1] = comb<F, T, V>(v1, qturn(u1, (3u + y + 2u * p1) & 3u), A, B);
  }
}

// x == 1: the pair is the aligned 2-vector (2q, 2q+1).
template <typename T, int F>
__global__ void __launch_bounds__(256) k_rot_pair1(typename Cx<T>::V* __restrict__ psi, uint64_t npairs, uint64_t z,
                                                   int y, T A, T B) {
  using V = typename Cx<T>::V;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t q = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; q < npairs; q += stride) {
    const uint64_t b = q << 1;
    const V u = psi[b], v = psi[b | 1ull];
    const unsigned p = par64(z & b);
    psi[b] = comb<F, T, V>(u, qturn(v, (3u + 3u * y + 2u * p) & 3u), A, B);
    psi[b | 1ull] = comb<F, T, V>(v, qturn(u, (3u + y + 2u * p) & 3u), A, B);
  }
}

// x == 0: diagonal phase, out[b] = A u + B i^{3+2par} u.
template <typename T, int F>
__global__ void __launch_bounds__(256) k_rot_diag(typename Cx<T>::V* __restrict__ psi, uint64_t N, uint64_t z, T A,
                                                  T B) {
  using V = typename Cx<T>::V;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t b = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; b < N; b += stride) {
    const V u = psi[b];
    psi[b] = comb<F, T, V>(u, qturn(u, (3u + 2u * par64(z & b)) & 3u), A, B);
  }
}

// ---------------------------------------------------------------------------
// fused rotations in a shared-memory tile
//
// A tile is the 2^s amplitudes whose bits outside the tile bit set S are fixed
// (S holds the union of the pass's X supports plus low bits for coalescing).
// The tile is read once, all m rotations act on it in shared memory (the part
// of z outside S only flips the sign class of the whole tile), and it is
// written once.

// One rotation of a fused pass on the staged tile.
template <int F, typename T>
__device__ __forceinline__ void tile_rot(typename Cx<T>::V* tile, const TileRot& R, unsigned pout, unsigned tsize, T A,
                                         T B) {
  using V = typename Cx<T>::V;
  if (R.hl < 0) {
    for (unsigned j = threadIdx.x; j < tsize; j += blockDim.x) {
      const unsigned p = (__popc(R.zl & j) + pout) & 1u;
      const V u = tile[j];
      tile[j] = comb<F, T, V>(u, qturn(u, (3u + 2u * p) & 3u), A, B);
    }
  } else {
    const unsigned hmask = (1u << R.hl) - 1u;
    for (unsigned q = threadIdx.x; q < (tsize >> 1); q += blockDim.x) {
      const unsigned j = ((q >> R.hl) << (R.hl + 1)) | (q & hmask);
      const unsigned jp = j ^ R.xl;
      const unsigned p = (__popc(R.zl & j) + pout) & 1u;
      const V u = tile[j], v = tile[jp];
      tile[j] = comb<F, T, V>(u, qturn(v, (3u + 3u * R.y + 2u * p) & 3u), A, B);
      tile[jp] = comb<F, T, V>(v, qturn(u, (3u + R.y + 2u * p) & 3u), A, B);
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(256) k_tile(typename Cx<T>::V* __restrict__ psi, int n,
                                              const __grid_constant__ TileArgs a) {
  using V = typename Cx<T>::V;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  V* tile = reinterpret_cast<V*>(smem_raw);
  uint64_t* hitab = reinterpret_cast<uint64_t*>(tile + (1 << a.s));
  const int s = a.s, l = a.l;
  const unsigned tsize = 1u << s, lmask = (1u << l) - 1u;
  for (int j = threadIdx.x; j < (1 << a.nhi); j += blockDim.x) {
    uint64_t off = 0;
    for (int i = 0; i < a.nhi; ++i)
      if ((j >> i) & 1) off |= 1ull << a.pos[i];
    hitab[j] = off;
  }
  const uint64_t ntiles = 1ull << (n - s);
  for (uint64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    uint64_t base = t;
    for (int i = 0; i < s; ++i) base = ins0(base, a.sbits[i]);
    __syncthreads();
#pragma unroll 8
    for (unsigned j = threadIdx.x; j < tsize; j += blockDim.x) tile[j] = psi[base | hitab[j >> l] | (j & lmask)];
    __syncthreads();
    for (int r = 0; r < a.m; ++r) {
      const TileRot R = a.r[r];
      const unsigned pout = par64(R.zout & base);
      const T A = (T)R.A, B = (T)R.B;
      if (R.form == FORM_A1)
        tile_rot<FORM_A1, T>(tile, R, pout, tsize, A, B);
      else if (R.form == FORM_B1)
        tile_rot<FORM_B1, T>(tile, R, pout, tsize, A, B);
      else
        tile_rot<FORM_AB, T>(tile, R, pout, tsize, A, B);
      __syncthreads();
    }
    for (unsigned j = threadIdx.x; j < tsize; j += blockDim.x) psi[base | hitab[j >> l] | (j & lmask)] = tile[j];
  }
}

// ---------------------------------------------------------------------------
// sparse composite block
//
// The composite of the block's rotations restricted to its support qubits is
// the identity except on a few "active" support patterns; only those
// amplitudes are read and written.  One thread per assignment of the
// non-support bits ("outside index").  The arguments hold M - I, so each output
// is v_r + sum_k (M - I)_rk v_k: the rounding then scales with the (small)
// change rather than with the amplitude, which keeps complex64 states close to
// unit norm.  REALM: M is real.  REALST: the state is real (imaginary parts are
// exactly zero and stay zero), so only real parts are read and written.

template <int NR>
struct SpK {
  int u, nr, nzc, pad;
  int supp[kSparseMaxSupp];
  uint64_t pat[NR];
  uint64_t zc[2];
  double2 M[kSparseMaxCls][NR][NR];
  double2 Q[kSparseMaxCls][NR][NR];
};

__device__ __forceinline__ uint64_t sp_base(uint64_t o, const int* supp, int u) {
  for (int i = 0; i < u; ++i) o = ins0(o, supp[i]);
  return o;
}

template <int NR>
__device__ __forceinline__ unsigned sp_class(const SpK<NR>& a, uint64_t base) {
  unsigned cls = 0;
  if (a.nzc > 0) cls = par64(a.zc[0] & base);
  if (a.nzc > 1) cls |= par64(a.zc[1] & base) << 1;
  return cls;
}

template <typename T, int NR, bool REALM, bool REALST>
__global__ void __launch_bounds__(256) k_sparse(typename Cx<T>::V* __restrict__ psi, int n,
                                                const __grid_constant__ SpK<NR> a) {
  using V = typename Cx<T>::V;
  __shared__ V M[kSparseMaxCls][NR][NR];
  for (int i = threadIdx.x; i < kSparseMaxCls * NR * NR; i += blockDim.x) {
    const int c = i / (NR * NR), r = (i / NR) % NR, k = i % NR;
    V m;
    m.x = (T)a.M[c][r][k].x;
    m.y = (T)a.M[c][r][k].y;
    M[c][r][k] = m;
  }
  __syncthreads();
  const uint64_t nout = 1ull << (n - a.u);
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  T* pr = reinterpret_cast<T*>(psi);
  for (uint64_t o = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; o < nout; o += stride) {
    const uint64_t base = sp_base(o, a.supp, a.u);
    const unsigned cls = sp_class(a, base);
    V v[NR];
#pragma unroll
    for (int r = 0; r < NR; ++r) {
      if (r < a.nr) {
        if (REALST) {
          v[r].x = pr[2 * (base | a.pat[r])];
          v[r].y = 0;
        } else {
          v[r] = psi[base | a.pat[r]];
        }
      }
    }
#pragma unroll
    for (int r = 0; r < NR; ++r) {
      if (r < a.nr) {
        T ox = v[r].x, oy = v[r].y;
#pragma unroll
        for (int k = 0; k < NR; ++k) {
          if (k < a.nr) {
            const V m = M[cls][r][k];
            ox = fma(m.x, v[k].x, ox);
            if (!REALST) oy = fma(m.x, v[k].y, oy);
            if (!REALM) {
              ox = fma(-m.y, v[k].y, ox);
              oy = fma(m.y, v[k].x, oy);
            }
          }
        }
        if (REALST) {
          pr[2 * (base | a.pat[r])] = ox;
        } else {
          V w;
          w.x = ox;
          w.y = oy;
          psi[base | a.pat[r]] = w;
        }
      }
    }
  }
}

// ---------------------------------------------------------------------------
// expectation value, pair form
//
// For an X group g (x != 0) and the pair (b, b xor x) with b's pivot bit clear,
// w = conj(psi[b xor x]) psi[b]; the pair's contribution from term t is
//   2 c_t (-1)^{y/2} s_t(b) Re w          (y even)
//   2 c_t (-1)^{(y+1)/2} s_t(b) Im w      (y odd),
// s_t(b) = (-1)^{popc(z_t & b)}.  Terms are packed four per chunk with a 16-entry
// table over their sign pattern, so a chunk costs one lookup and one or two
// FMAs per pair.  The diagonal group (x = 0) uses |psi_b|^2 and c_t.

template <typename T>
__global__ void __launch_bounds__(256) k_expect(const typename Cx<T>::V* __restrict__ psi, int n,
                                                const ExpGroup* __restrict__ groups, int ngroups,
                                                const ExpChunk* __restrict__ chunks, double* partials,
                                                unsigned* counter, double* out) {
  using V = typename Cx<T>::V;
  const uint64_t hmask = (1ull << (n - 1)) - 1ull;
  const uint64_t total = (uint64_t)ngroups << (n - 1);
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  double acc = 0.0;
  // complex64: pair products and table weights in FP32, folded into the FP64
  // accumulator every 32 pairs (no per-pair FP64 conversions)
  float facc = 0.f;
  int nf = 0;
  for (uint64_t f = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; f < total; f += stride) {
    const int g = (int)(f >> (n - 1));
    const uint64_t p = f & hmask;
    const ExpGroup G = groups[g];
    if (G.h < 0) {
      const uint64_t b0 = p << 1;
      const V u0 = psi[b0], u1 = psi[b0 | 1ull];
      for (int c = 0; c < G.nchunk; ++c) {
        const ExpChunk* C = chunks + G.chunk0 + c;
        unsigned i0 = 0, i1 = 0;
#pragma unroll
        for (int t = 0; t < kChunkTerms; ++t) {
          const uint64_t zt = C->z[t];
          const unsigned pb = par64(zt & b0);
          i0 |= pb << t;
          i1 |= (pb ^ (unsigned)(zt & 1ull)) << t;
        }
        if constexpr (sizeof(T) == 4) {
          facc = fmaf(C->ftab[i0].x, fmaf(u0.x, u0.x, u0.y * u0.y), facc);
          facc = fmaf(C->ftab[i1].x, fmaf(u1.x, u1.x, u1.y * u1.y), facc);
        } else {
          acc = fma(C->tab[i0].x, fma((double)u0.x, u0.x, (double)u0.y * u0.y), acc);
          acc = fma(C->tab[i1].x, fma((double)u1.x, u1.x, (double)u1.y * u1.y), acc);
        }
      }
    } else {
      const uint64_t b = ins0(p, G.h);
      const V u = psi[b], v = psi[b ^ G.x];
      T rew = 0, imw = 0;
      if (G.flags & 1) rew = fma(u.x, v.x, u.y * v.y);
      if (G.flags & 2) imw = fma(u.y, v.x, -u.x * v.y);
      for (int c = 0; c < G.nchunk; ++c) {
        const ExpChunk* C = chunks + G.chunk0 + c;
        unsigned idx = 0;
#pragma unroll
        for (int t = 0; t < kChunkTerms; ++t) idx |= par64(C->z[t] & b) << t;
        if constexpr (sizeof(T) == 4) {
          const float2 D = C->ftab[idx];
          if (G.flags & 1) facc = fmaf(D.x, rew, facc);
          if (G.flags & 2) facc = fmaf(D.y, imw, facc);
        } else {
          const double2 D = C->tab[idx];
          if (G.flags & 1) acc = fma(D.x, rew, acc);
          if (G.flags & 2) acc = fma(D.y, imw, acc);
        }
      }
    }
    if constexpr (sizeof(T) == 4) {
      if (++nf == 32) {
        acc += (double)facc;
        facc = 0.f;
        nf = 0;
      }
    }
  }
  acc += (double)facc;
  grid_finish(acc, partials, counter, out);
}

// Tiled form for n > 10: a CTA takes tiles of 256 x P pairs of one X group
// (P = 4; 8 was slower for complex64 at 28 qubits), reads the group's descriptor
// once per tile, and every thread issues the loads of its P pairs before using
// them (P times the loads in flight of the flat loop).  A group of one term
// (flags bit 2: its table is +-tab[0]) puts the sign on the amplitude and the
// weight on the tile's sum, so a pair costs two multiply-adds.
template <typename T> struct ExpTile {
  static constexpr int P = 4;
  static constexpr int LOG = 10;  // log2(256 P)
};
constexpr int kExpTileLogMax = 10;

template <typename T>
__global__ void __launch_bounds__(256) k_expect_tiled(const typename Cx<T>::V* __restrict__ psi, int n,
                                                      const ExpGroup* __restrict__ groups, int ngroups,
                                                      const ExpChunk* __restrict__ chunks, double* partials,
                                                      unsigned* counter, double* out) {
  using V = typename Cx<T>::V;
  constexpr int kExpPairs = ExpTile<T>::P, kExpTileLog = ExpTile<T>::LOG;
  const int tb = n - 1 - kExpTileLog;  // log2(tiles per group)
  const uint64_t ntiles = (uint64_t)ngroups << tb;
  double acc = 0.0;
  float facc = 0.f;  // complex64: FP32 sums folded into acc once per tile
  for (uint64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int g = (int)(tile >> tb);
    const uint64_t p0 = ((tile & ((1ull << tb) - 1)) << kExpTileLog) + threadIdx.x;
    const ExpGroup G = groups[g];
    if (G.h < 0) {  // x = 0: |psi_b|^2 of both amplitudes of each pair
#pragma unroll
      for (int k = 0; k < kExpPairs; ++k) {
        const uint64_t b0 = (p0 + 256 * k) << 1;
        const V u0 = psi[b0], u1 = psi[b0 | 1ull];
        for (int c = 0; c < G.nchunk; ++c) {
          const ExpChunk* C = chunks + G.chunk0 + c;
          unsigned i0 = 0, i1 = 0;
#pragma unroll
          for (int t = 0; t < kChunkTerms; ++t) {
            const uint64_t zt = C->z[t];
            const unsigned pb = par64(zt & b0);
            i0 |= pb << t;
            i1 |= (pb ^ (unsigned)(zt & 1ull)) << t;
          }
          if constexpr (sizeof(T) == 4) {
            facc = fmaf(C->ftab[i0].x, fmaf(u0.x, u0.x, u0.y * u0.y), facc);
            facc = fmaf(C->ftab[i1].x, fmaf(u1.x, u1.x, u1.y * u1.y), facc);
          } else {
            acc = fma(C->tab[i0].x, fma((double)u0.x, u0.x, (double)u0.y * u0.y), acc);
            acc = fma(C->tab[i1].x, fma((double)u1.x, u1.x, (double)u1.y * u1.y), acc);
          }
        }
      }
    } else {
      uint64_t b[kExpPairs];
      V u[kExpPairs], v[kExpPairs];
#pragma unroll
      for (int k = 0; k < kExpPairs; ++k) {
        b[k] = ins0(p0 + 256 * k, G.h);
        u[k] = psi[b[k]];
        v[k] = psi[b[k] ^ G.x];
      }
      if (G.flags & 4) {  // one term: D = (-1)^{popc(z & b)} tab[0]
        const ExpChunk* C = chunks + G.chunk0;
        const uint64_t z = C->z[0];
        T gr = T(0), gi = T(0);
#pragma unroll
        for (int k = 0; k < kExpPairs; ++k) {
          const unsigned sg = par64(z & b[k]);
          const T ux = sg ? -u[k].x : u[k].x, uy = sg ? -u[k].y : u[k].y;
          if (G.flags & 1) gr = fma(ux, v[k].x, fma(uy, v[k].y, gr));
          if (G.flags & 2) gi = fma(uy, v[k].x, fma(-ux, v[k].y, gi));
        }
        if constexpr (sizeof(T) == 4) {
          const float2 D = C->ftab[0];
          facc = fmaf(D.x, gr, fmaf(D.y, gi, facc));
        } else {
          const double2 D = C->tab[0];
          acc = fma(D.x, gr, fma(D.y, gi, acc));
        }
      } else {
#pragma unroll
        for (int k = 0; k < kExpPairs; ++k) {
          T rew = 0, imw = 0;
          if (G.flags & 1) rew = fma(u[k].x, v[k].x, u[k].y * v[k].y);
          if (G.flags & 2) imw = fma(u[k].y, v[k].x, -u[k].x * v[k].y);
          for (int c = 0; c < G.nchunk; ++c) {
            const ExpChunk* C = chunks + G.chunk0 + c;
            unsigned idx = 0;
#pragma unroll
            for (int t = 0; t < kChunkTerms; ++t) idx |= par64(C->z[t] & b[k]) << t;
            if constexpr (sizeof(T) == 4) {
              const float2 D = C->ftab[idx];
              if (G.flags & 1) facc = fmaf(D.x, rew, facc);
              if (G.flags & 2) facc = fmaf(D.y, imw, facc);
            } else {
              const double2 D = C->tab[idx];
              if (G.flags & 1) acc = fma(D.x, rew, acc);
              if (G.flags & 2) acc = fma(D.y, imw, acc);
            }
          }
        }
      }
    }
    if constexpr (sizeof(T) == 4) {
      acc += (double)facc;
      facc = 0.f;
    }
  }
  grid_finish(acc, partials, counter, out);
}

// ---------------------------------------------------------------------------
// lam = H psi (gather form) fused with out[0] = Re <psi|lam>, out[1] = <psi|psi>
//
// lam[c] = sum_g D_g(c xor x_g) psi[c xor x_g], D_g(b) = sum_t c_t i^{y_t} s_t(b);
// D is read from the same 16-entry chunk tables (real part from even-y terms,
// imaginary part from odd-y terms).

template <typename T>
__global__ void __launch_bounds__(256) k_hpsi(const typename Cx<T>::V* __restrict__ psi,
                                              typename Cx<T>::V* __restrict__ lam, int n,
                                              const ExpGroup* __restrict__ groups, int ngroups,
                                              const ExpChunk* __restrict__ chunks, double* partials,
                                              unsigned* counter, double* out) {
  using V = typename Cx<T>::V;
  const uint64_t N = 1ull << n;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  double acc = 0.0, nrm = 0.0;
  for (uint64_t cidx = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; cidx < N; cidx += stride) {
    double lx = 0.0, ly = 0.0;
    for (int g = 0; g < ngroups; ++g) {
      const ExpGroup G = groups[g];
      const uint64_t b = cidx ^ G.x;
      const V v = psi[b];
      double dx = 0.0, dy = 0.0;
      for (int c = 0; c < G.nchunk; ++c) {
        const ExpChunk* C = chunks + G.chunk0 + c;
        unsigned idx = 0;
#pragma unroll
        for (int t = 0; t < kChunkTerms; ++t) idx |= par64(C->z[t] & b) << t;
        const double2 D = C->tab[idx];
        dx += D.x;
        dy += D.y;
      }
      const double vx = (double)v.x, vy = (double)v.y;
      lx = fma(dx, vx, lx);
      ly = fma(dx, vy, ly);
      if (G.flags & 2) {
        lx = fma(-dy, vy, lx);
        ly = fma(dy, vx, ly);
      }
    }
    const V u = psi[cidx];
    acc = fma((double)u.x, lx, fma((double)u.y, ly, acc));
    nrm = fma((double)u.x, (double)u.x, fma((double)u.y, (double)u.y, nrm));
    V w;
    w.x = (T)lx;
    w.y = (T)ly;
    lam[cidx] = w;
  }
  grid_finish2(acc, nrm, partials, counter, out);
}

// ---------------------------------------------------------------------------
// tiled H|psi>: lam[c] = sum_g D_g(c xor x_g) psi[c xor x_g], out[0] = Re <psi|lam>,
// out[1] = <psi|psi>.
//
// Output tiles are 2^TB contiguous amplitudes (TB = 8 + log2 E; each of the 256
// threads owns E of them: c = tid + 256 k).  For every class of groups sharing
// the high part xh of their X mask, the partner tile (tile xor xh) is staged in
// shared memory once and all groups of the class read it there.  For element k
// the partner index inside the tile is (tid ^ xl) | ((k ^ xl >> 8) << 8), and the
// sign pattern of the group's terms splits into a per-thread part and a part
// that depends on k only, so the inner loop is an XOR, a table load and an FMA.
// REALST: psi is real and every D is real, so only real parts are used.
// For float states each class's contribution is summed in FP32 and folded into
// FP64 accumulators once per class.

template <typename T> struct WTab;
template <> struct WTab<double> { using C = WChunk; using V2 = double2; };
template <> struct WTab<float> { using C = WChunkF; using V2 = float2; };

template <typename T, int E, bool REALST>
__global__ void __launch_bounds__(256) k_hpsi_tiled(const typename Cx<T>::V* __restrict__ psi,
                                                    typename Cx<T>::V* __restrict__ lam, int n,
                                                    const HClass* __restrict__ classes, int nclasses,
                                                    const HGroup* __restrict__ groups,
                                                    const typename WTab<T>::C* __restrict__ chunks,
                                                    double* partials, unsigned* counter, double* out) {
  using V = typename Cx<T>::V;
  constexpr int TB = (E == 1) ? 8 : (E == 2) ? 9 : (E == 4) ? 10 : (E == 8) ? 11 : 12;
  constexpr int KB = TB - 8;  // bits of k
  extern __shared__ __align__(16) unsigned char smem_raw[];
  V* tile = reinterpret_cast<V*>(smem_raw);
  const unsigned tid = threadIdx.x;
  const uint64_t ntiles = 1ull << (n - TB);
  double acc_e = 0.0, acc_n = 0.0;
  for (uint64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    double lx[E], ly[E];
#pragma unroll
    for (int k = 0; k < E; ++k) lx[k] = ly[k] = 0.0;
    for (int ci = 0; ci < nclasses; ++ci) {
      const HClass C = classes[ci];
      const uint64_t pt = t ^ C.xh;
      __syncthreads();
#pragma unroll
      for (int k = 0; k < E; ++k) tile[tid + 256u * k] = psi[(pt << TB) + tid + 256u * k];
      __syncthreads();
      T fx[E], fy[E];
#pragma unroll
      for (int k = 0; k < E; ++k) fx[k] = fy[k] = 0;
      for (int g = C.g0; g < C.g1; ++g) {
        const HGroup G = groups[g];
        const unsigned xl = (unsigned)(G.x & ((1ull << TB) - 1ull));
        const unsigned xlo = xl & 255u, xhi = xl >> 8;
        T dx[E], dy[E];
        // the first table initialises D (no add of zero), later tables add to it
        for (int c = 0; c < G.nchunk; ++c) {
          const typename WTab<T>::C* W = chunks + G.chunk0 + c;
          unsigned ith = 0, col[KB > 0 ? KB : 1];
#pragma unroll
          for (int j = 0; j < (KB > 0 ? KB : 1); ++j) col[j] = 0;
#pragma unroll
          for (int q = 0; q < kWideTerms; ++q) {
            const uint64_t z = W->z[q];
            const unsigned hp = par64((z >> TB) & pt);
            const unsigned tp = (unsigned)__popc((unsigned)z & 255u & (tid ^ xlo)) & 1u;
            ith |= (hp ^ tp) << q;
#pragma unroll
            for (int j = 0; j < KB; ++j) col[j] |= (unsigned)((z >> (8 + j)) & 1ull) << q;
          }
#pragma unroll
          for (int k = 0; k < E; ++k) {
            unsigned idx = ith;
            const unsigned kk = (unsigned)k ^ xhi;
#pragma unroll
            for (int j = 0; j < KB; ++j)
              if ((kk >> j) & 1u) idx ^= col[j];
            const typename WTab<T>::V2 d = W->tab[idx];
            if (c == 0) {
              dx[k] = d.x;
              if (!REALST) dy[k] = d.y;
            } else {
              dx[k] += d.x;
              if (!REALST) dy[k] += d.y;
            }
          }
        }
#pragma unroll
        for (int k = 0; k < E; ++k) {
          const V v = tile[(tid ^ xlo) | ((((unsigned)k ^ xhi)) << 8)];
          fx[k] = fma(dx[k], v.x, fx[k]);
          if (!REALST) {
            fy[k] = fma(dx[k], v.y, fy[k]);
            if (G.odd) {
              fx[k] = fma(-dy[k], v.y, fx[k]);
              fy[k] = fma(dy[k], v.x, fy[k]);
            }
          }
        }
      }
#pragma unroll
      for (int k = 0; k < E; ++k) {
        lx[k] += (double)fx[k];
        if (!REALST) ly[k] += (double)fy[k];
      }
    }
#pragma unroll
    for (int k = 0; k < E; ++k) {
      const uint64_t cidx = (t << TB) + tid + 256u * k;
      const V u = psi[cidx];
      acc_e = fma((double)u.x, lx[k], fma((double)u.y, ly[k], acc_e));
      acc_n = fma((double)u.x, (double)u.x, fma((double)u.y, (double)u.y, acc_n));
      V w;
      w.x = (T)lx[k];
      w.y = (T)ly[k];
      lam[cidx] = w;
    }
  }
  grid_finish2(acc_e, acc_n, partials, counter, out);
}

// ---------------------------------------------------------------------------
// tiled H|psi> for a real complex128 state and real D_g, double-single arithmetic
//
// GB300 executes FP64 FMAs at 1/58 of the FP32 rate, and this gather needs one
// multiply-add per (X group, amplitude).  Here each staged partner amplitude
// and each table value is split into a pair of floats (hi + lo, ~48 bits), the
// product D * v is formed exactly in its leading part (p = dh*vh and its FMA
// residual) plus the cross terms dh*vl + dl*vh, and it is accumulated with an
// error-free TwoSum into a (hi, lo) float pair per output amplitude.  Per
// operation the relative error is about 2^-46; the pair is renormalised once per
// class and converted to FP64 when the tile is written.  Groups with more than
// eight terms contribute one product per eight-term table.

// The _rn intrinsics keep the compiler from contracting or reassociating the
// error-free transformations.
__device__ __forceinline__ void ds_mad(float& ah, float& al, float dh, float dl, float vh, float vl) {
  const float p = __fmul_rn(dh, vh);
  float e = fmaf(dh, vh, -p);
  e = fmaf(dh, vl, e);
  e = fmaf(dl, vh, e);
  const float s = __fadd_rn(ah, p);
  const float bp = __fsub_rn(s, ah);
  const float err = __fadd_rn(__fsub_rn(ah, __fsub_rn(s, bp)), __fsub_rn(p, bp));
  al = __fadd_rn(al, __fadd_rn(err, e));
  ah = s;
}

__global__ void __launch_bounds__(256) k_split_ds(const double2* __restrict__ psi, float2* __restrict__ out,
                                                  uint64_t N) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < N; i += stride) {
    const double v = psi[i].x;
    const float h = __double2float_rn(v);
    out[i] = make_float2(h, __double2float_rn(v - (double)h));
  }
}

// Tiles of 2^12 amplitudes; thread t owns c = t + 256 k (k < 16).  For group
// g with low X bits xl = xlo + 256 xhi the partner of element k is
// (t ^ xlo) + 256 (k ^ xhi), and the sign-pattern index of a table is
//   hp (tile part, uniform) ^ nl[(t^xlo) & 15] ^ nh[(t^xlo) >> 4] ^ kx[k].
__global__ void __launch_bounds__(256) k_hpsi_ds(const double2* __restrict__ psi, const float2* __restrict__ split,
                                                 double2* __restrict__ lam, int n,
                                                 const HClass* __restrict__ classes, int nclasses,
                                                 const HGroup* __restrict__ groups,
                                                 const WChunkS* __restrict__ chunks, double* partials,
                                                 unsigned* counter, double* out) {
  constexpr int TB = 12, E = 16;
  __shared__ float2 tile[1 << TB];
  const unsigned tid = threadIdx.x;
  const uint64_t ntiles = 1ull << (n - TB);
  double acc_e = 0.0, acc_n = 0.0;
  for (uint64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    float ah[E], al[E];
#pragma unroll
    for (int k = 0; k < E; ++k) ah[k] = al[k] = 0.f;
    for (int ci = 0; ci < nclasses; ++ci) {
      const HClass C = classes[ci];
      const uint64_t pt = t ^ C.xh;
      __syncthreads();
#pragma unroll
      for (int k = 0; k < E; ++k) tile[tid + 256u * k] = split[(pt << TB) + tid + 256u * k];
      __syncthreads();
      for (int g = C.g0; g < C.g1; ++g) {
        const HGroup G = groups[g];
        const unsigned xlo = (unsigned)G.x & 255u;
        const unsigned tx = tid ^ xlo;
        for (int c = 0; c < G.nchunk; ++c) {
          const WChunkS* W = chunks + G.chunk0 + c;
          unsigned ith = (unsigned)W->nl[tx & 15u] ^ (unsigned)W->nh[tx >> 4];
#pragma unroll
          for (int q = 0; q < kWideTerms; ++q) ith ^= par64(W->zh[q] & pt) << q;
          const uint4 kxw = *reinterpret_cast<const uint4*>(W->kx);
          const unsigned kw[4] = {kxw.x, kxw.y, kxw.z, kxw.w};
          const unsigned xhi = ((unsigned)G.x >> 8) & 15u;
#pragma unroll
          for (int k = 0; k < E; ++k) {
            const unsigned idx = ith ^ ((kw[k >> 2] >> (8 * (k & 3))) & 255u);
            const float2 d = W->tab[idx];
            const float2 v = tile[tx | (((unsigned)k ^ xhi) << 8)];
            ds_mad(ah[k], al[k], d.x, d.y, v.x, v.y);
          }
        }
      }
#pragma unroll
      for (int k = 0; k < E; ++k) {  // renormalise the pair once per class
        const float s = __fadd_rn(ah[k], al[k]);
        al[k] = __fsub_rn(al[k], __fsub_rn(s, ah[k]));
        ah[k] = s;
      }
    }
#pragma unroll
    for (int k = 0; k < E; ++k) {
      const uint64_t cidx = (t << TB) + tid + 256u * k;
      const double lx = (double)ah[k] + (double)al[k];
      const double2 u = psi[cidx];
      acc_e = fma(u.x, lx, acc_e);
      acc_n = fma(u.x, u.x, acc_n);
      lam[cidx] = make_double2(lx, 0.0);
    }
  }
  grid_finish2(acc_e, acc_n, partials, counter, out);
}

// ---------------------------------------------------------------------------
// adjoint step for one rotation: out = Im <lam|P|psi> (pre-rotation values),
// then psi and lam both get the rotation given in the arguments (the host passes
// -theta, i.e. exp(+i theta P)).
//
// Over the pair (b, b'): <lam|P|psi> gets i^y s(b) [(-1)^y conj(lam_b) psi_b' +
// conj(lam_b') psi_b].

template <typename T, int F>
__global__ void __launch_bounds__(256) k_adj_rot(typename Cx<T>::V* __restrict__ psi,
                                                 typename Cx<T>::V* __restrict__ lam, int n, uint64_t x, uint64_t z,
                                                 int h, int y, T A, T B, double* partials, unsigned* counter,
                                                 double* out) {
  using V = typename Cx<T>::V;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  double acc = 0.0;
  const unsigned ym = (unsigned)y & 3u;
  if (x == 0ull) {
    const uint64_t N = 1ull << n;
    for (uint64_t b = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; b < N; b += stride) {
      const V u = psi[b], p = lam[b];
      const unsigned pb = par64(z & b);
      // Im(conj(p) s u)
      const double im = fma((double)p.x, (double)u.y, -(double)p.y * (double)u.x);
      acc += flip(im, pb);
      psi[b] = comb<F, T, V>(u, qturn(u, (3u + 2u * pb) & 3u), A, B);
      lam[b] = comb<F, T, V>(p, qturn(p, (3u + 2u * pb) & 3u), A, B);
    }
  } else {
    const uint64_t npairs = 1ull << (n - 1);
    for (uint64_t q = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; q < npairs; q += stride) {
      const uint64_t b = ins0(q, h), bp = b ^ x;
      const V u = psi[b], v = psi[bp], p = lam[b], r = lam[bp];
      const unsigned pb = par64(z & b);
      double val;
      if ((ym & 1u) == 0u) {
        // Im z1 + Im z2, z1 = conj(p) v, z2 = conj(r) u
        const double i1 = fma((double)p.x, (double)v.y, -(double)p.y * (double)v.x);
        const double i2 = fma((double)r.x, (double)u.y, -(double)r.y * (double)u.x);
        val = flip(i1 + i2, (ym >> 1) ^ pb);
      } else {
        // Re z2 - Re z1
        const double r1 = fma((double)p.x, (double)v.x, (double)p.y * (double)v.y);
        const double r2 = fma((double)r.x, (double)u.x, (double)r.y * (double)u.y);
        val = flip(r2 - r1, ((ym >> 1) & 1u) ^ pb);
      }
      acc += val;
      psi[b] = comb<F, T, V>(u, qturn(v, (3u + 3u * y + 2u * pb) & 3u), A, B);
      psi[bp] = comb<F, T, V>(v, qturn(u, (3u + y + 2u * pb) & 3u), A, B);
      lam[b] = comb<F, T, V>(p, qturn(r, (3u + 3u * y + 2u * pb) & 3u), A, B);
      lam[bp] = comb<F, T, V>(r, qturn(p, (3u + y + 2u * pb) & 3u), A, B);
    }
  }
  grid_finish(acc, partials, counter, out);
}

// adjoint step for a sparse block: out = Im <lam|Q|psi>, then psi <- M psi,
// lam <- M lam on the active rows (the arguments hold M - I for the block's
// inverse composite M).  RQ: M is real and Q = i * (real matrix), the case of
// every fermionic excitation block, where Im <lam|Q|psi> = sum Qi_rk Re(conj(lam_r) psi_k).
template <typename T, int NR, bool RQ, bool REALST>
__global__ void __launch_bounds__(256) k_adj_sparse(typename Cx<T>::V* __restrict__ psi,
                                                    typename Cx<T>::V* __restrict__ lam, int n,
                                                    const __grid_constant__ SpK<NR> a, double* partials,
                                                    unsigned* counter, double* out) {
  using V = typename Cx<T>::V;
  __shared__ V M[kSparseMaxCls][NR][NR];
  __shared__ double2 Q[kSparseMaxCls][NR][NR];
  for (int i = threadIdx.x; i < kSparseMaxCls * NR * NR; i += blockDim.x) {
    const int c = i / (NR * NR), r = (i / NR) % NR, k = i % NR;
    V m;
    m.x = (T)a.M[c][r][k].x;
    m.y = (T)a.M[c][r][k].y;
    M[c][r][k] = m;
    Q[c][r][k] = a.Q[c][r][k];
  }
  __syncthreads();
  const uint64_t nout = 1ull << (n - a.u);
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  T* pr = reinterpret_cast<T*>(psi);
  T* lr = reinterpret_cast<T*>(lam);
  double acc = 0.0;
  for (uint64_t o = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; o < nout; o += stride) {
    const uint64_t base = sp_base(o, a.supp, a.u);
    const unsigned cls = sp_class(a, base);
    V v[NR], w[NR];
#pragma unroll
    for (int r = 0; r < NR; ++r) {
      if (r < a.nr) {
        const uint64_t idx = base | a.pat[r];
        if (REALST) {
          v[r].x = pr[2 * idx];
          w[r].x = lr[2 * idx];
          v[r].y = w[r].y = 0;
        } else {
          v[r] = psi[idx];
          w[r] = lam[idx];
        }
      }
    }
#pragma unroll
    for (int r = 0; r < NR; ++r) {
      if (r < a.nr) {
        if (RQ) {
          // Re <lam_r|Qi v>, in the state's precision (FP64 accumulation across items)
          T sx = 0, sy = 0;
#pragma unroll
          for (int k = 0; k < NR; ++k)
            if (k < a.nr) {
              const T qi = (T)Q[cls][r][k].y;
              sx = fma(qi, v[k].x, sx);
              if (!REALST) sy = fma(qi, v[k].y, sy);
            }
          acc += (double)fma(w[r].x, sx, REALST ? (T)0 : w[r].y * sy);
        } else {
          double qx = 0.0, qy = 0.0;
#pragma unroll
          for (int k = 0; k < NR; ++k) {
            if (k < a.nr) {
              const double2 q = Q[cls][r][k];
              qx = fma(q.x, (double)v[k].x, fma(-q.y, (double)v[k].y, qx));
              qy = fma(q.x, (double)v[k].y, fma(q.y, (double)v[k].x, qy));
            }
          }
          acc = fma((double)w[r].x, qy, fma(-(double)w[r].y, qx, acc));
        }
      }
    }
#pragma unroll
    for (int r = 0; r < NR; ++r) {
      if (r < a.nr) {
        T ox = v[r].x, oy = v[r].y, px = w[r].x, py = w[r].y;
#pragma unroll
        for (int k = 0; k < NR; ++k) {
          if (k < a.nr) {
            const V m = M[cls][r][k];
            ox = fma(m.x, v[k].x, ox);
            px = fma(m.x, w[k].x, px);
            if (!REALST) {
              oy = fma(m.x, v[k].y, oy);
              py = fma(m.x, w[k].y, py);
            }
            if (!RQ) {
              ox = fma(-m.y, v[k].y, ox);
              oy = fma(m.y, v[k].x, oy);
              px = fma(-m.y, w[k].y, px);
              py = fma(m.y, w[k].x, py);
            }
          }
        }
        const uint64_t idx = base | a.pat[r];
        if (REALST) {
          pr[2 * idx] = ox;
          lr[2 * idx] = px;
        } else {
          V o1, o2;
          o1.x = ox;
          o1.y = oy;
          o2.x = px;
          o2.y = py;
          psi[idx] = o1;
          lam[idx] = o2;
        }
      }
    }
  }
  grid_finish(acc, partials, counter, out);
}

int g_sms = 0;

int sm_count() {
  if (g_sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&g_sms, cudaDevAttrMultiProcessorCount, dev);
    if (g_sms <= 0) g_sms = 152;
  }
  return g_sms;
}

unsigned grid_for(uint64_t work, int per_sm) {
  const uint64_t cap = (uint64_t)sm_count() * per_sm;
  uint64_t g = (work + 255) / 256;
  if (g > cap) g = cap;
  if (g < 1) g = 1;
  return (unsigned)g;
}

thread_local uint64_t t_launches = 0;

// opt-in per-launch event timing
struct ProfRec {
  unsigned kind;
  cudaEvent_t a, b;
};
thread_local unsigned t_prof_mask = 0;
thread_local std::vector<ProfRec> t_prof;
thread_local std::vector<cudaEvent_t> t_ev_pool;
thread_local size_t t_prof_used = 0;

cudaEvent_t pool_event(size_t i) {
  while (t_ev_pool.size() <= i) {
    cudaEvent_t e;
    cudaEventCreate(&e);
    t_ev_pool.push_back(e);
  }
  return t_ev_pool[i];
}

}  // namespace

void count_launch() { ++t_launches; }

// Records the start event of a launch of `kind` (if profiled); returns a slot.
int prof_pre(unsigned kind, cudaStream_t s) {
  if (!(t_prof_mask & kind)) return -1;
  ProfRec r{kind, pool_event(2 * t_prof_used), pool_event(2 * t_prof_used + 1)};
  ++t_prof_used;
  cudaEventRecord(r.a, s);
  t_prof.push_back(r);
  return (int)t_prof.size() - 1;
}

void prof_post(int slot, cudaStream_t s) {
  if (slot >= 0) cudaEventRecord(t_prof[slot].b, s);
}

int profile_begin(unsigned mask) {
  t_prof.clear();
  t_prof_used = 0;
  t_prof_mask = mask;
  return 0;
}

cudaError_t profile_read(unsigned mask, uint64_t* launches, double* total_ms) {
  uint64_t n = 0;
  double ms = 0.0;
  for (const ProfRec& r : t_prof) {
    if (!(r.kind & mask)) continue;
    cudaError_t e = cudaEventSynchronize(r.b);
    if (e != cudaSuccess) return e;
    float f = 0.f;
    e = cudaEventElapsedTime(&f, r.a, r.b);
    if (e != cudaSuccess) return e;
    ms += f;
    ++n;
  }
  if (launches) *launches = n;
  if (total_ms) *total_ms = ms;
  return cudaSuccess;
}

void profile_end() {
  t_prof_mask = 0;
  t_prof.clear();
  t_prof_used = 0;
}

int reduce_blocks(int n, qf_dtype) {
  const uint64_t cap = (uint64_t)sm_count() * 4;
  uint64_t g = ((1ull << n) / 2 + 255) / 256;
  if (g > cap) g = cap;
  if (g < 1) g = 1;
  return (int)g;
}

cudaError_t launch_zero_and_set(void* psi, int n, qf_dtype dt, uint64_t det, cudaStream_t s) {
  return launch_zero_and_set_count(psi, 1ull << n, dt, det, s);
}

cudaError_t launch_zero_and_set_count(void* psi, uint64_t N, qf_dtype dt, uint64_t det, cudaStream_t s) {
  const int prof_slot_ = prof_pre(QF_K_SET, s);
  const unsigned g = grid_for(N, 8);
  if (dt == QF_C128)
    k_zero_and_set<double2><<<g, 256, 0, s>>>(static_cast<double2*>(psi), N, det);
  else
    k_zero_and_set<float2><<<g, 256, 0, s>>>(static_cast<float2*>(psi), N, det);
  prof_post(prof_slot_, s);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_gather(const void* src, qf_dtype dt, const int64_t* idx, int count, bool packed, bool ds,
                          double* out, cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  if (ds && (dt != QF_C128 || !packed)) return cudaErrorInvalidValue;
  const unsigned g = (unsigned)((count + 255) / 256);
  if (ds)
    k_gather_ds<<<g, 256, 0, s>>>(static_cast<const float4*>(src), idx, count, out);
  else if (dt == QF_C128)
    k_gather<double2><<<g, 256, 0, s>>>(static_cast<const double2*>(src), idx, count, packed ? 1 : 0, out);
  else
    k_gather<float2><<<g, 256, 0, s>>>(static_cast<const float2*>(src), idx, count, packed ? 1 : 0, out);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_scale(void* psi, int n, qf_dtype dt, double scale, cudaStream_t s) {
  const int prof_slot_ = prof_pre(QF_K_SET, s);
  const uint64_t N = 1ull << n;
  const unsigned g = grid_for(N, 8);
  if (dt == QF_C128)
    k_scale<double><<<g, 256, 0, s>>>(static_cast<double2*>(psi), N, scale);
  else
    k_scale<float><<<g, 256, 0, s>>>(static_cast<float2*>(psi), N, (float)scale);
  prof_post(prof_slot_, s);
  count_launch();
  return cudaGetLastError();
}

template <typename T, int F>
static void rot_impl_f(void* psi, int n, const RotArgs& a, cudaStream_t s) {
  using V = typename Cx<T>::V;
  V* p = static_cast<V*>(psi);
  const uint64_t N = 1ull << n;
  if (a.x == 0ull) {
    k_rot_diag<T, F><<<grid_for(N, 8), 256, 0, s>>>(p, N, a.z, (T)a.A, (T)a.B);
  } else if (a.h == 0) {
    k_rot_pair1<T, F><<<grid_for(N / 2, 8), 256, 0, s>>>(p, N / 2, a.z, a.y, (T)a.A, (T)a.B);
  } else {
    k_rot_pair2<T, F><<<grid_for(N / 4, 8), 256, 0, s>>>(p, N / 4, a.x, a.z, a.h, a.y, (T)a.A, (T)a.B);
  }
}

template <typename T>
static void rot_impl(void* psi, int n, const RotArgs& a, cudaStream_t s) {
  if (a.form == FORM_A1)
    rot_impl_f<T, FORM_A1>(psi, n, a, s);
  else if (a.form == FORM_B1)
    rot_impl_f<T, FORM_B1>(psi, n, a, s);
  else
    rot_impl_f<T, FORM_AB>(psi, n, a, s);
}

cudaError_t launch_rot(void* psi, int n, qf_dtype dt, const RotArgs& a, cudaStream_t s) {
  const int prof_slot_ = prof_pre(QF_K_ROT, s);
  if (dt == QF_C128)
    rot_impl<double>(psi, n, a, s);
  else
    rot_impl<float>(psi, n, a, s);
  prof_post(prof_slot_, s);
  count_launch();
  return cudaGetLastError();
}

template <typename T>
static cudaError_t tile_impl(void* psi, int n, const TileArgs& a, cudaStream_t s) {
  using V = typename Cx<T>::V;
  const size_t smem = (sizeof(V) << a.s) + (sizeof(uint64_t) << a.nhi);
  static bool attr_set = false;
  if (!attr_set) {
    cudaFuncSetAttribute(k_tile<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    attr_set = true;
  }
  const uint64_t ntiles = 1ull << (n - a.s);
  int per_sm = 4;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_tile<T>, 256, smem);
  uint64_t g = (uint64_t)sm_count() * (uint64_t)std::max(1, per_sm);
  if (g > ntiles) g = ntiles;
  k_tile<T><<<(unsigned)g, 256, smem, s>>>(static_cast<V*>(psi), n, a);
  return cudaGetLastError();
}

cudaError_t launch_tile(void* psi, int n, qf_dtype dt, const TileArgs& a, cudaStream_t s) {
  const int prof_slot_ = prof_pre(QF_K_TILE, s);
  cudaError_t e = dt == QF_C128 ? tile_impl<double>(psi, n, a, s) : tile_impl<float>(psi, n, a, s);
  prof_post(prof_slot_, s);
  count_launch();
  return e;
}

template <int NR>
static SpK<NR> compact(const SparseArgs& a) {
  SpK<NR> k;
  memset(&k, 0, sizeof(k));
  k.u = a.u;
  k.nr = a.nr;
  k.nzc = a.nzc;
  for (int i = 0; i < kSparseMaxSupp; ++i) k.supp[i] = a.supp[i];
  for (int r = 0; r < NR && r < a.nr; ++r) k.pat[r] = a.pat[r];
  k.zc[0] = a.zc[0];
  k.zc[1] = a.zc[1];
  for (int c = 0; c < kSparseMaxCls; ++c)
    for (int r = 0; r < NR && r < a.nr; ++r)
      for (int q = 0; q < NR && q < a.nr; ++q) {
        k.M[c][r][q] = a.M[c][r][q];
        k.Q[c][r][q] = a.Q[c][r][q];
      }
  return k;
}

bool sparse_m_real(const SparseArgs& a) {
  for (int c = 0; c < a.ncls; ++c)
    for (int r = 0; r < a.nr; ++r)
      for (int k = 0; k < a.nr; ++k)
        if (a.M[c][r][k].y != 0.0) return false;
  return true;
}

bool sparse_q_imag(const SparseArgs& a) {
  for (int c = 0; c < a.ncls; ++c)
    for (int r = 0; r < a.nr; ++r)
      for (int k = 0; k < a.nr; ++k)
        if (a.Q[c][r][k].x != 0.0) return false;
  return true;
}

template <typename T, int NR>
static void sparse_fwd(void* psi, int n, const SparseArgs& a, bool realst, cudaStream_t s) {
  using V = typename Cx<T>::V;
  const SpK<NR> k = compact<NR>(a);
  const unsigned g = grid_for(1ull << (n - a.u), 8);
  V* p = static_cast<V*>(psi);
  const bool rm = sparse_m_real(a);
  if (rm && realst)
    k_sparse<T, NR, true, true><<<g, 256, 0, s>>>(p, n, k);
  else if (rm)
    k_sparse<T, NR, true, false><<<g, 256, 0, s>>>(p, n, k);
  else
    k_sparse<T, NR, false, false><<<g, 256, 0, s>>>(p, n, k);
}

template <typename T, int NR>
static void sparse_adj(void* psi, void* lam, int n, const SparseArgs& a, bool realst, double* partials,
                       unsigned* counter, double* out, int nblocks, cudaStream_t s) {
  using V = typename Cx<T>::V;
  const SpK<NR> k = compact<NR>(a);
  V* p = static_cast<V*>(psi);
  V* l = static_cast<V*>(lam);
  const bool rq = sparse_m_real(a) && sparse_q_imag(a);
  if (rq && realst)
    k_adj_sparse<T, NR, true, true><<<nblocks, 256, 0, s>>>(p, l, n, k, partials, counter, out);
  else if (rq)
    k_adj_sparse<T, NR, true, false><<<nblocks, 256, 0, s>>>(p, l, n, k, partials, counter, out);
  else
    k_adj_sparse<T, NR, false, false><<<nblocks, 256, 0, s>>>(p, l, n, k, partials, counter, out);
}

template <typename T>
static void sparse_fwd_nr(void* psi, int n, const SparseArgs& a, bool realst, cudaStream_t s) {
  if (a.nr <= 2)
    sparse_fwd<T, 2>(psi, n, a, realst, s);
  else if (a.nr <= 4)
    sparse_fwd<T, 4>(psi, n, a, realst, s);
  else
    sparse_fwd<T, 8>(psi, n, a, realst, s);
}

template <typename T>
static void sparse_adj_nr(void* psi, void* lam, int n, const SparseArgs& a, bool realst, double* partials,
                          unsigned* counter, double* out, int nblocks, cudaStream_t s) {
  if (a.nr <= 2)
    sparse_adj<T, 2>(psi, lam, n, a, realst, partials, counter, out, nblocks, s);
  else if (a.nr <= 4)
    sparse_adj<T, 4>(psi, lam, n, a, realst, partials, counter, out, nblocks, s);
  else
    sparse_adj<T, 8>(psi, lam, n, a, realst, partials, counter, out, nblocks, s);
}

cudaError_t launch_sparse(void* psi, int n, qf_dtype dt, const SparseArgs& a, bool realst, cudaStream_t s) {
  const int prof_slot_ = prof_pre(QF_K_SPARSE, s);
  if (dt == QF_C128)
    sparse_fwd_nr<double>(psi, n, a, realst, s);
  else
    sparse_fwd_nr<float>(psi, n, a, realst, s);
  prof_post(prof_slot_, s);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_expect(const void* psi, int n, qf_dtype dt, const ExpGroup* groups, int ngroups,
                          const ExpChunk* chunks, double* partials, unsigned* counter, double* out, int nblocks,
                          cudaStream_t s) {
  const int prof_slot_ = prof_pre(QF_K_EXPECT, s);
  const bool tiled = n > kExpTileLogMax;  // at least one whole tile per group
  if (dt == QF_C128) {
    if (tiled)
      k_expect_tiled<double><<<nblocks, 256, 0, s>>>(static_cast<const double2*>(psi), n, groups, ngroups, chunks,
                                                     partials, counter, out);
    else
      k_expect<double><<<nblocks, 256, 0, s>>>(static_cast<const double2*>(psi), n, groups, ngroups, chunks,
                                               partials, counter, out);
  } else {
    if (tiled)
      k_expect_tiled<float><<<nblocks, 256, 0, s>>>(static_cast<const float2*>(psi), n, groups, ngroups, chunks,
                                                    partials, counter, out);
    else
      k_expect<float><<<nblocks, 256, 0, s>>>(static_cast<const float2*>(psi), n, groups, ngroups, chunks,
                                              partials, counter, out);
  }
  prof_post(prof_slot_, s);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_hpsi(const void* psi, void* lam, int n, qf_dtype dt, const ExpGroup* groups, int ngroups,
                        const ExpChunk* chunks, double* partials, unsigned* counter, double* out, int nblocks,
                        cudaStream_t s) {
  const int prof_slot_ = prof_pre(QF_K_HPSI, s);
  if (dt == QF_C128)
    k_hpsi<double><<<nblocks, 256, 0, s>>>(static_cast<const double2*>(psi), static_cast<double2*>(lam), n, groups,
                                           ngroups, chunks, partials, counter, out);
  else
    k_hpsi<float><<<nblocks, 256, 0, s>>>(static_cast<const float2*>(psi), static_cast<float2*>(lam), n, groups,
                                          ngroups, chunks, partials, counter, out);
  prof_post(prof_slot_, s);
  count_launch();
  return cudaGetLastError();
}

template <typename T, int E>
static cudaError_t hpsi_tiled_e(const void* psi, void* lam, int n, bool realst, const HClass* classes, int nclasses,
                                const HGroup* groups, const void* chunks, double* partials, unsigned* counter,
                                double* out, int nblocks, cudaStream_t s) {
  using V = typename Cx<T>::V;
  using C = typename WTab<T>::C;
  const size_t smem = sizeof(V) * 256 * E;
  const uint64_t ntiles = 1ull << (n - (8 + (E == 1 ? 0 : E == 2 ? 1 : E == 4 ? 2 : E == 8 ? 3 : 4)));
  // persistent grid: exactly the blocks that are resident at once (a partial
  // second wave would leave most SMs idle at the end)
  int per_sm = 1;
  if (realst)
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_hpsi_tiled<T, E, true>, 256, smem);
  else
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_hpsi_tiled<T, E, false>, 256, smem);
  if (per_sm < 1) per_sm = 1;
  uint64_t cap = (uint64_t)sm_count() * (uint64_t)per_sm;
  if (cap > (uint64_t)nblocks) cap = (uint64_t)nblocks;
  unsigned g = (unsigned)std::min<uint64_t>(ntiles, cap);
  if (realst) {
    cudaFuncSetAttribute(k_hpsi_tiled<T, E, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_hpsi_tiled<T, E, true><<<g, 256, smem, s>>>(static_cast<const V*>(psi), static_cast<V*>(lam), n, classes,
                                                  nclasses, groups, static_cast<const C*>(chunks), partials,
                                                  counter, out);
  } else {
    cudaFuncSetAttribute(k_hpsi_tiled<T, E, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_hpsi_tiled<T, E, false><<<g, 256, smem, s>>>(static_cast<const V*>(psi), static_cast<V*>(lam), n, classes,
                                                   nclasses, groups, static_cast<const C*>(chunks), partials,
                                                   counter, out);
  }
  return cudaGetLastError();
}

template <typename T>
static cudaError_t hpsi_tiled_t(const void* psi, void* lam, int n, int tb, bool realst, const HClass* classes,
                                int nclasses, const HGroup* groups, const void* chunks, double* partials,
                                unsigned* counter, double* out, int nblocks, cudaStream_t s) {
  switch (tb) {
    case 8: return hpsi_tiled_e<T, 1>(psi, lam, n, realst, classes, nclasses, groups, chunks, partials, counter, out, nblocks, s);
    case 9: return hpsi_tiled_e<T, 2>(psi, lam, n, realst, classes, nclasses, groups, chunks, partials, counter, out, nblocks, s);
    case 10: return hpsi_tiled_e<T, 4>(psi, lam, n, realst, classes, nclasses, groups, chunks, partials, counter, out, nblocks, s);
    case 11: return hpsi_tiled_e<T, 8>(psi, lam, n, realst, classes, nclasses, groups, chunks, partials, counter, out, nblocks, s);
    case 12: return hpsi_tiled_e<T, 16>(psi, lam, n, realst, classes, nclasses, groups, chunks, partials, counter, out, nblocks, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_hpsi_tiled(const void* psi, void* lam, int n, qf_dtype dt, int tb, bool realst,
                              const HClass* classes, int nclasses, const HGroup* groups, const void* chunks,
                              double* partials, unsigned* counter, double* out, int nblocks, cudaStream_t s) {
  const int prof_slot_ = prof_pre(QF_K_HPSI, s);
  cudaError_t e = (dt == QF_C128)
                      ? hpsi_tiled_t<double>(psi, lam, n, tb, realst, classes, nclasses, groups, chunks, partials,
                                             counter, out, nblocks, s)
                      : hpsi_tiled_t<float>(psi, lam, n, tb, realst, classes, nclasses, groups, chunks, partials,
                                            counter, out, nblocks, s);
  prof_post(prof_slot_, s);
  count_launch();
  return e;
}

cudaError_t launch_hpsi_ds(const void* psi, void* lam, void* split, int n, const HClass* classes, int nclasses,
                           const HGroup* groups, const WChunkS* chunks, double* partials, unsigned* counter,
                           double* out, int nblocks, cudaStream_t s) {
  const int prof_slot_ = prof_pre(QF_K_HPSI, s);
  const uint64_t N = 1ull << n;
  k_split_ds<<<grid_for(N, 8), 256, 0, s>>>(static_cast<const double2*>(psi), static_cast<float2*>(split), N);
  int per_sm = 1;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_hpsi_ds, 256, 0);
  if (per_sm < 1) per_sm = 1;
  uint64_t cap = (uint64_t)sm_count() * (uint64_t)per_sm;
  if (cap > (uint64_t)nblocks) cap = (uint64_t)nblocks;
  const unsigned g = (unsigned)std::min<uint64_t>(1ull << (n - 12), cap);
  k_hpsi_ds<<<g, 256, 0, s>>>(static_cast<const double2*>(psi), static_cast<const float2*>(split),
                              static_cast<double2*>(lam), n, classes, nclasses, groups, chunks, partials, counter,
                              out);
  prof_post(prof_slot_, s);
  count_launch();
  count_launch();
  return cudaGetLastError();
}

template <typename T, int F>
static void adj_rot_f(void* psi, void* lam, int n, const RotArgs& a, double* partials, unsigned* counter, double* out,
                      int nblocks, cudaStream_t s) {
  using V = typename Cx<T>::V;
  k_adj_rot<T, F><<<nblocks, 256, 0, s>>>(static_cast<V*>(psi), static_cast<V*>(lam), n, a.x, a.z, a.h, a.y, (T)a.A,
                                          (T)a.B, partials, counter, out);
}

template <typename T>
static void adj_rot_t(void* psi, void* lam, int n, const RotArgs& a, double* partials, unsigned* counter, double* out,
                      int nblocks, cudaStream_t s) {
  if (a.form == FORM_A1)
    adj_rot_f<T, FORM_A1>(psi, lam, n, a, partials, counter, out, nblocks, s);
  else if (a.form == FORM_B1)
    adj_rot_f<T, FORM_B1>(psi, lam, n, a, partials, counter, out, nblocks, s);
  else
    adj_rot_f<T, FORM_AB>(psi, lam, n, a, partials, counter, out, nblocks, s);
}

cudaError_t launch_adj_rot(void* psi, void* lam, int n, qf_dtype dt, const RotArgs& a, double* partials,
                           unsigned* counter, double* out, int nblocks, cudaStream_t s) {
  const int prof_slot_ = prof_pre(QF_K_ADJ_ROT, s);
  if (dt == QF_C128)
    adj_rot_t<double>(psi, lam, n, a, partials, counter, out, nblocks, s);
  else
    adj_rot_t<float>(psi, lam, n, a, partials, counter, out, nblocks, s);
  prof_post(prof_slot_, s);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_adj_sparse(void* psi, void* lam, int n, qf_dtype dt, const SparseArgs& a, bool realst,
                              double* partials, unsigned* counter, double* out, int nblocks, cudaStream_t s) {
  const int prof_slot_ = prof_pre(QF_K_ADJ_SPARSE, s);
  if (dt == QF_C128)
    sparse_adj_nr<double>(psi, lam, n, a, realst, partials, counter, out, nblocks, s);
  else
    sparse_adj_nr<float>(psi, lam, n, a, realst, partials, counter, out, nblocks, s);
  prof_post(prof_slot_, s);
  count_launch();
  return cudaGetLastError();
}

}  // namespace qf

extern "C" uint64_t qf_kernel_launches(int reset) {
  const uint64_t v = qf::t_launches;
  if (reset) qf::t_launches = 0;
  return v;
}
