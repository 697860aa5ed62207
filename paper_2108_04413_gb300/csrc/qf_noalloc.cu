// qf_expectation_noalloc: an expectation-value entry point that allocates no
// device memory.
//
// Who needs it: callers that cannot call cudaMalloc.  Examples are a host
// application whose device memory is fully reserved by another allocator (a
// framework's caching pool, a serving process with a fixed HBM budget), and a
// latency-critical loop that must not take cudaMalloc's implicit device-wide
// synchronisation.  qf_expectation needs a qf_state handle, and creating one
// allocates reduction scratch and the grouped term tables.  This entry point
// instead reads amplitudes the caller already owns and keeps its scratch in
// the fixed-size device array below.  That array is part of the library image,
// so every GPU that loads libqf holds it (1 MiB) until the process exits.
//
// The scratch holds the reduction counter, the result, the per-block partial
// sums and the X-mask group tables (at most QF_NOALLOC_MAX_TERMS terms).  All
// calls share it and it keeps the previous call's contents: the counter is
// cleared at the start of each call, and everything else is overwritten before
// it is read.  Two calls whose GPU work overlapped would race on the array, so
// each call holds a process-wide lock from its table upload until its stream
// has synchronised: calls from several host threads run one after another.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <mutex>
#include <string>

#include "qf_internal.h"

namespace {

constexpr size_t kOffCounter = 0;
constexpr size_t kOffOut = 256;
constexpr size_t kMaxPartials = 1024;
constexpr size_t kOffPartials = 512;
constexpr size_t kOffGroups = kOffPartials + kMaxPartials * sizeof(double);
constexpr size_t kOffChunks =
    (kOffGroups + QF_NOALLOC_MAX_TERMS * sizeof(qf::ExpGroup) + 255) / 256 * 256;
constexpr size_t kNeeded = kOffChunks + QF_NOALLOC_MAX_TERMS * sizeof(qf::ExpChunk);
static_assert(kNeeded <= QF_NOALLOC_SCRATCH_BYTES, "scratch layout exceeds the stated size");

// The device scratch.  Host code must not use this name as an address: on the
// host it is only a stand-in symbol, so its device address is looked up with
// cudaGetSymbolAddress (once per device) and passed to the kernels.
static __device__ __align__(256) unsigned char g_scratch[QF_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
unsigned char* g_dev_addr[kMaxDevices] = {};
std::mutex g_mu;  // guards g_dev_addr and the host staging tables

// Host staging for the group tables (static: no heap allocation per call).
qf::ExpGroup h_groups[QF_NOALLOC_MAX_TERMS];
qf::ExpChunk h_chunks[QF_NOALLOC_MAX_TERMS];
uint32_t h_order[QF_NOALLOC_MAX_TERMS];

qf_status nfail(qf_status s, const char* msg, cudaError_t e = cudaSuccess) {
  std::string m(msg);
  if (e != cudaSuccess) {
    m += ": ";
    m += cudaGetErrorString(e);
  }
  qf::set_last_error(m);
  return s;
}

int popc(uint64_t v) { return __builtin_popcountll(v); }
int hibit(uint64_t v) { return v ? 63 - __builtin_clzll(v) : -1; }

// Device address of g_scratch on the current device, looked up on first use.
qf_status scratch_address(unsigned char** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return nfail(QF_ECUDA, "cudaGetDevice failed", e);
  if (dev < 0 || dev >= kMaxDevices) return nfail(QF_EINVAL, "device ordinal too large for the no-alloc table");
  if (!g_dev_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess || !p) return nfail(QF_ECUDA, "cudaGetSymbolAddress(scratch) failed", e);
    g_dev_addr[dev] = static_cast<unsigned char*>(p);
  }
  *out = g_dev_addr[dev];
  return QF_OK;
}

// Group the terms by X mask into the static host tables (same weights as the
// pair-form expectation kernel: 2 c (-1)^{y/2} on Re w for even y, 2 c (-1)^{(y+1)/2}
// on Im w for odd y, c on |psi|^2 for the diagonal group).
void build_tables(const qf_term* terms, size_t nt, int* ngroups, int* nchunks) {
  for (size_t i = 0; i < nt; ++i) h_order[i] = (uint32_t)i;
  std::sort(h_order, h_order + nt, [&](uint32_t a, uint32_t b) {
    return terms[a].x < terms[b].x || (terms[a].x == terms[b].x && a < b);
  });
  int ng = 0, nc = 0;
  size_t i = 0;
  while (i < nt) {
    size_t j = i;
    while (j < nt && terms[h_order[j]].x == terms[h_order[i]].x) ++j;
    qf::ExpGroup& g = h_groups[ng++];
    g.x = terms[h_order[i]].x;
    g.h = hibit(g.x);
    g.chunk0 = nc;
    g.nchunk = 0;
    g.flags = 0;
    for (size_t k = i; k < j; k += qf::kChunkTerms) {
      qf::ExpChunk& c = h_chunks[nc++];
      ++g.nchunk;
      const int cnt = (int)std::min<size_t>(qf::kChunkTerms, j - k);
      for (int t = 0; t < qf::kChunkTerms; ++t) c.z[t] = (t < cnt) ? terms[h_order[k + t]].z : 0ull;
      for (int pat = 0; pat < (1 << qf::kChunkTerms); ++pat) {
        double ex = 0.0, ey = 0.0;
        for (int t = 0; t < cnt; ++t) {
          const qf_term& T = terms[h_order[k + t]];
          const int y = popc(T.x & T.z) & 3;
          const double cv = ((pat >> t) & 1) ? -T.coeff : T.coeff;
          if ((y & 1) == 0)
            ex += (g.x == 0 ? 1.0 : 2.0) * cv * ((y == 2) ? -1.0 : 1.0);
          else
            ey += 2.0 * cv * ((y == 1) ? -1.0 : 1.0);
        }
        c.tab[pat] = make_double2(ex, ey);
        c.ftab[pat] = make_float2((float)ex, (float)ey);
      }
      for (int t = 0; t < cnt; ++t) {
        const qf_term& T = terms[h_order[k + t]];
        g.flags |= (popc(T.x & T.z) & 1) ? 2 : 1;
      }
    }
    if (j - i == 1) g.flags |= 4;  // a single term (the same flag as the state path's plans)
    i = j;
  }
  *ngroups = ng;
  *nchunks = nc;
}

}  // namespace

extern "C" qf_status qf_expectation_noalloc(const void* amplitudes, int n, qf_dtype dtype, void* stream,
                                            const qf_term* terms, size_t n_terms, double* re, double* im) {
  if (!amplitudes || !re) return nfail(QF_EINVAL, "NULL argument");
  if (n < 1 || n > QF_MAX_QUBITS) return nfail(QF_EINVAL, "qubit count outside 1..QF_MAX_QUBITS");
  if (dtype != QF_C128 && dtype != QF_C64) return nfail(QF_EINVAL, "unknown dtype");
  if (reinterpret_cast<uintptr_t>(amplitudes) & 15u) return nfail(QF_EINVAL, "amplitudes not 16-byte aligned");
  if (n_terms > QF_NOALLOC_MAX_TERMS)
    return nfail(QF_EINVAL, "too many terms for the allocation-free path (limit QF_NOALLOC_MAX_TERMS)");
  if (n_terms && !terms) return nfail(QF_EINVAL, "term list is NULL");
  const uint64_t lim = (1ull << n) - 1ull;
  for (size_t k = 0; k < n_terms; ++k)
    if ((terms[k].x & ~lim) || (terms[k].z & ~lim))
      return nfail(QF_EINVAL, "Pauli mask has a bit at or above the qubit count");
  if (im) *im = 0.0;
  if (n_terms == 0) {
    *re = 0.0;
    return QF_OK;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  std::lock_guard<std::mutex> lock(g_mu);
  unsigned char* base = nullptr;
  qf_status st = scratch_address(&base);
  if (st != QF_OK) return st;
  int ng = 0, nc = 0;
  build_tables(terms, n_terms, &ng, &nc);
  unsigned* counter = reinterpret_cast<unsigned*>(base + kOffCounter);
  double* out = reinterpret_cast<double*>(base + kOffOut);
  double* partials = reinterpret_cast<double*>(base + kOffPartials);
  qf::ExpGroup* d_groups = reinterpret_cast<qf::ExpGroup*>(base + kOffGroups);
  qf::ExpChunk* d_chunks = reinterpret_cast<qf::ExpChunk*>(base + kOffChunks);
  cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(unsigned), s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_groups, h_groups, ng * sizeof(qf::ExpGroup), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_chunks, h_chunks, nc * sizeof(qf::ExpChunk), cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return nfail(QF_ECUDA, "copy into the no-alloc scratch failed", e);
  int nb = qf::reduce_blocks(n, dtype);
  if (nb > (int)kMaxPartials) nb = (int)kMaxPartials;
  e = qf::launch_expect(amplitudes, n, dtype, d_groups, ng, d_chunks, partials, counter, out, nb, s);
  if (e != cudaSuccess) return nfail(QF_ECUDA, "expectation kernel launch failed", e);
  double v = 0.0;
  e = cudaMemcpyAsync(&v, out, sizeof(double), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return nfail(QF_ECUDA, "reading the no-alloc result failed", e);
  *re = v;
  return QF_OK;
}
