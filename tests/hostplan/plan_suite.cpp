// Runs the C ABI's calls on the CUDA test double (cuda_stub.cpp) and prints, per
// call, its status and the digest of everything it would have sent to the
// device.  Inputs are raw arrays written by tests/test_hostplan_cpu.py:
//   plan_suite <dir>          every case, one line each
//   plan_suite <dir> layout   sizeof and field offsets of qf::SparseArgs
//   plan_suite <dir> tables   the same for qf::ExpGroup and qf::ExpChunk
//   plan_suite <dir> secblk   the same for qf::SecBlk, and the coefficient record length
//   plan_suite <dir> runitems <n> <det>   the part-local sweep's items per run for
//                             terms_ri.bin / ansatz_ri.bin / t_ri.bin
#include <cstddef>
#include <cstdio>
#include <cstdlib>
#include <limits>
#include <string>
#include <thread>
#include <vector>

#include "qf.h"
#include "qf_internal.h"

namespace stub {
extern thread_local uint64_t digest;
extern thread_local size_t copies, h2d_bytes;
void reset();
size_t live_bytes();
void dump_live();
}  // namespace stub

static std::string g_dir;

template <typename T>
static std::vector<T> load(const char* name) {
  const std::string path = g_dir + "/" + name;
  FILE* f = std::fopen(path.c_str(), "rb");
  if (!f) {
    std::fprintf(stderr, "missing input %s\n", path.c_str());
    std::exit(2);
  }
  std::fseek(f, 0, SEEK_END);
  const long n = std::ftell(f);
  std::fseek(f, 0, SEEK_SET);
  std::vector<T> v((size_t)n / sizeof(T));
  if (std::fread(v.data(), sizeof(T), v.size(), f) != v.size()) std::exit(2);
  std::fclose(f);
  return v;
}

static void report(const std::string& name, qf_status s) {
  std::printf("%s %d %zu %zu %016llx\n", name.c_str(), (int)s, stub::copies, stub::h2d_bytes,
              (unsigned long long)stub::digest);
  if (s != QF_OK) std::printf("#error %s: %s\n", name.c_str(), qf_last_error());
  stub::reset();
}

static qf_state* make(int n, qf_dtype dt) {
  qf_state* st = nullptr;
  if (qf_state_create(n, dt, nullptr, nullptr, 0, &st) != QF_OK) {
    std::printf("#error create: %s\n", qf_last_error());
    std::exit(3);
  }
  return st;
}

int main(int argc, char** argv) {
  if (argc < 2) return 1;
  g_dir = argv[1];
  if (argc > 2 && std::string(argv[2]) == "layout") {
    using qf::SparseArgs;
    std::printf("%zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %d %d %d\n", sizeof(SparseArgs), offsetof(SparseArgs, u),
                offsetof(SparseArgs, nr), offsetof(SparseArgs, ncls), offsetof(SparseArgs, nzc),
                offsetof(SparseArgs, supp), offsetof(SparseArgs, pat), offsetof(SparseArgs, zc),
                offsetof(SparseArgs, M), offsetof(SparseArgs, Q), qf::kSparseMaxSupp, qf::kSparseMaxRows,
                qf::kSparseMaxCls);
    return 0;
  }
  if (argc > 2 && std::string(argv[2]) == "tables") {
    using qf::ExpChunk;
    using qf::ExpGroup;
    std::printf("%zu %zu %zu %zu %zu %zu %zu %zu %zu %d\n", sizeof(ExpGroup), offsetof(ExpGroup, x),
                offsetof(ExpGroup, nchunk), offsetof(ExpGroup, chunk0), sizeof(ExpChunk), offsetof(ExpChunk, z),
                offsetof(ExpChunk, tab), offsetof(ExpChunk, ftab), (size_t)(1 << qf::kChunkTerms), qf::kChunkTerms);
    return 0;
  }
  if (argc > 2 && std::string(argv[2]) == "secblk") {
    using qf::SecBlk;
    std::printf("%zu %zu %zu %zu %d %zu\n", sizeof(SecBlk), offsetof(SecBlk, pat), offsetof(SecBlk, zc),
                offsetof(SecBlk, nzc), qf::kSmallCoef, offsetof(SecBlk, m));
    return 0;
  }
  if (argc > 5 && std::string(argv[2]) == "footprint") {
    // device bytes a handle holds after one evaluation of terms_fp.bin / ansatz_fp.bin / t_fp.bin
    const auto T = load<qf_term>("terms_fp.bin");
    const auto A = load<qf_arot>("ansatz_fp.bin");
    const auto t = load<double>("t_fp.bin");
    const size_t before = stub::live_bytes();
    qf_state* st = make(std::atoi(argv[3]), std::string(argv[4]) == "c64" ? QF_C64 : QF_C128);
    std::vector<double> grad(t.size());
    double energy = 0;
    const qf_status s = qf_energy_grad(st, std::strtoull(argv[5], nullptr, 0), A.data(), A.size(), t.data(),
                                       t.size(), T.data(), T.size(), &energy, grad.data());
    if (s != QF_OK) {
      std::printf("#error footprint: %s\n", qf_last_error());
      return 4;
    }
    std::printf("%zu\n", stub::live_bytes() - before);
    if (std::getenv("QF_STUB_LIST")) stub::dump_live();
    qf_state_destroy(st);
    return 0;
  }
  if (argc > 5 && std::string(argv[2]) == "circuit") {
    // rot_c.bin applied to |det> (or, with "trotter", terms_c.bin evolved for time 0.3 in 3 steps);
    // prints the scale the state keeps aside
    const int n = std::atoi(argv[3]);
    qf_state* st = make(n, std::string(argv[5]) == "c64" ? QF_C64 : QF_C128);
    qf_set_basis(st, std::strtoull(argv[4], nullptr, 0));
    qf_status s;
    if (argc > 6 && std::string(argv[6]) == "trotter") {
      const auto H = load<qf_term>("terms_c.bin");
      s = qf_trotter(st, H.data(), H.size(), 0.3, 3);
    } else {
      const auto R = load<qf_rot>("rot_c.bin");
      s = qf_apply_circuit(st, R.data(), R.size());
    }
    double scale = 0;
    qf_state_info(st, nullptr, nullptr, nullptr, &scale);
    std::printf("%d %.17g\n", (int)s, scale);
    qf_state_destroy(st);
    return 0;
  }
  if (argc > 4 && std::string(argv[2]) == "runitems") {
    const auto T = load<qf_term>("terms_ri.bin");
    const auto A = load<qf_arot>("ansatz_ri.bin");
    const auto t = load<double>("t_ri.bin");
    qf_state* st = make(std::atoi(argv[3]), QF_C128);
    std::vector<double> grad(t.size());
    double energy = 0;
    const qf_status s = qf_energy_grad(st, std::strtoull(argv[4], nullptr, 0), A.data(), A.size(), t.data(),
                                       t.size(), T.data(), T.size(), &energy, grad.data());
    if (s != QF_OK) {
      std::printf("#error runitems: %s\n", qf_last_error());
      return 4;
    }
    size_t nr = 0;
    qf_sweep_run_items(st, nullptr, 0, &nr);
    std::vector<uint64_t> items(nr);
    qf_sweep_run_items(st, items.data(), nr, &nr);
    for (uint64_t v : items) std::printf("%llu\n", (unsigned long long)v);
    qf_state_destroy(st);
    return 0;
  }
  const auto T16 = load<qf_term>("terms16.bin");
  const auto A16 = load<qf_arot>("ansatz16.bin");
  auto t16 = load<double>("t16.bin");
  const auto R16 = load<qf_rot>("rot16.bin");
  const auto P16 = load<qf_arot>("pool16.bin");
  const auto D16 = load<uint64_t>("dets16.bin");
  const auto A10 = load<qf_arot>("ansatz10.bin");
  const auto t10 = load<double>("t10.bin");
  const auto T10 = load<qf_term>("terms10.bin");
  const auto R10 = load<qf_rot>("rot10.bin");
  const auto H10 = load<qf_term>("ham10.bin");
  const auto A8 = load<qf_arot>("ansatz8.bin");
  const auto t8 = load<double>("t8.bin");
  const auto T8 = load<qf_term>("terms8.bin");
  const std::string only = argc > 2 ? argv[2] : "";
  std::vector<double> g(4096), r(4096), gp(4096), es(16);
  double e = 0, re = 0, im = 0;
  stub::reset();
  if (only.empty() || only == "sector16") {
    qf_state* st = make(16, QF_C128);
    report("energy_grad.16q.cold", qf_energy_grad(st, 255, A16.data(), A16.size(), t16.data(), t16.size(),
                                                  T16.data(), T16.size(), &e, g.data()));
    // the first call also sets up the handle (compact layout, tables kept across plans);
    // from then on every rebuilt plan must send the device the same bytes
    for (const char* name : {"energy_grad.16q.rebuilt", "energy_grad.16q.rebuilt_again"}) {
      qf_state_clear_plans(st);
      stub::reset();
      report(name, qf_energy_grad(st, 255, A16.data(), A16.size(), t16.data(), t16.size(), T16.data(), T16.size(),
                                  &e, g.data()));
    }
    t16[0] += 0.01;
    report("energy_grad.16q.warm", qf_energy_grad(st, 255, A16.data(), A16.size(), t16.data(), t16.size(),
                                                  T16.data(), T16.size(), &e, g.data()));
    t16[0] -= 0.01;
    report("pool_gradients.16q", qf_pool_gradients(st, 255, A16.data(), A16.size(), t16.data(), t16.size(),
                                                   T16.data(), T16.size(), P16.data(), P16.size(), t16.size(), &e,
                                                   gp.data()));
    report("residuals.16q", qf_residuals(st, 255, A16.data(), A16.size(), t16.data(), t16.size(), T16.data(),
                                         T16.size(), D16.data(), D16.size(), &e, g.data(), r.data()));
    qf_set_basis(st, 255);
    stub::reset();
    report("apply_circuit.16q.ucc", qf_apply_circuit(st, R16.data(), R16.size()));
    report("expectation.16q", qf_expectation(st, T16.data(), T16.size(), &re, &im));
    qf_state_destroy(st);
  }
  if (only == "direct8" || only == "direct10") {  // a molecular sector evaluation: the direct tables
    const bool ten = only == "direct10";
    const auto A = load<qf_arot>(ten ? "ansatz10.bin" : "ansatz8.bin");
    const auto T = load<qf_term>(ten ? "terms10.bin" : "terms8.bin");
    const auto t = load<double>(ten ? "t10.bin" : "t8.bin");
    qf_state* st = make(ten ? 10 : 8, QF_C128);
    // (the 10-qubit ansatz file starts with a particle-number-changing rotation: skip it)
    const size_t skip = ten ? 1 : 0, npar = ten ? t.size() - 1 : t.size() / 4;
    std::vector<qf_arot> A2(A.begin() + skip, A.end());
    for (auto& a : A2) a.param -= (int32_t)skip;
    report(only == "direct8" ? "energy_grad.8q.direct" : "energy_grad.10q.direct",
           qf_energy_grad(st, ten ? 31 : 15, A2.data(), A2.size(), t.data() + skip, npar, T.data(), T.size(), &e,
                          g.data()));
    qf_state_destroy(st);
  }
  if (only == "errors") {  // rejected calls: their status, then a valid call on the same handle
    const size_t base = stub::live_bytes();
    qf_state* ref = make(16, QF_C128);
    qf_energy_grad(ref, 255, A16.data(), A16.size(), t16.data(), t16.size(), T16.data(), T16.size(), &e, g.data());
    const size_t clean = stub::live_bytes() - base;
    qf_state_destroy(ref);
    qf_state* st = make(16, QF_C128);
    std::vector<qf_term> Tbad(T16);
    Tbad[7].z |= 1ull << 16;  // a Pauli letter on a qubit the state does not have
    std::printf("#status mask %d\n", (int)qf_energy_grad(st, 255, A16.data(), A16.size(), t16.data(), t16.size(),
                                                         Tbad.data(), Tbad.size(), &e, g.data()));
    std::vector<qf_arot> Abad(A16);
    Abad[3].param = (int32_t)t16.size();  // a parameter index past the vector
    std::printf("#status param %d\n", (int)qf_energy_grad(st, 255, Abad.data(), Abad.size(), t16.data(),
                                                          t16.size(), T16.data(), T16.size(), &e, g.data()));
    std::vector<double> tbad(t16);
    tbad[5] = std::numeric_limits<double>::quiet_NaN();
    std::printf("#status angle %d\n", (int)qf_energy_grad(st, 255, A16.data(), A16.size(), tbad.data(),
                                                          tbad.size(), T16.data(), T16.size(), &e, g.data()));
    std::printf("#status det %d\n", (int)qf_energy_grad(st, 255ull | (1ull << 20), A16.data(), A16.size(),
                                                        t16.data(), t16.size(), T16.data(), T16.size(), &e,
                                                        g.data()));
    std::printf("#status null %d\n", (int)qf_energy_grad(st, 255, A16.data(), A16.size(), nullptr, t16.size(),
                                                         T16.data(), T16.size(), &e, g.data()));
    std::printf("#status valid %d\n", (int)qf_energy_grad(st, 255, A16.data(), A16.size(), t16.data(),
                                                          t16.size(), T16.data(), T16.size(), &e, g.data()));
    std::printf("#held %zu %zu\n", clean, stub::live_bytes() - base);
    qf_state_destroy(st);
  }
  if (only == "big28") {  // the 28-qubit random workload: a 4 GiB register, 500 rotations, 20000 terms
    const auto R = load<qf_rot>("rot28.bin");
    const auto H = load<qf_term>("ham28.bin");
    for (int d = 0; d < 2; ++d) {
      qf_state* st = make(28, d ? QF_C64 : QF_C128);
      qf_set_basis(st, (1ull << 14) - 1);
      stub::reset();
      report(std::string("apply_circuit.28q") + (d ? ".c64" : ".c128"), qf_apply_circuit(st, R.data(), R.size()));
      report(std::string("expectation.28q") + (d ? ".c64" : ".c128"),
             qf_expectation(st, H.data(), H.size(), &re, &im));
      qf_state_destroy(st);
    }
  }
  if (only == "threads") {  // one 16-qubit handle per host thread, evaluated at once
    auto one = [&](uint64_t* out, double scale) {
      stub::reset();
      std::vector<double> t(t16), gg(t16.size());
      for (double& v : t) v *= scale;
      double en = 0;
      qf_state* st = make(16, QF_C128);
      for (int rep = 0; rep < 3; ++rep)
        if (qf_energy_grad(st, 255, A16.data(), A16.size(), t.data(), t.size(), T16.data(), T16.size(), &en,
                           gg.data()) != QF_OK)
          std::printf("#error thread: %s\n", qf_last_error());
      qf_state_destroy(st);
      *out = stub::digest;
    };
    uint64_t serial[4], conc[4];
    for (int k = 0; k < 4; ++k) one(&serial[k], 1.0 + 0.1 * k);
    std::vector<std::thread> th;
    for (int k = 0; k < 4; ++k) th.emplace_back(one, &conc[k], 1.0 + 0.1 * k);
    for (auto& x : th) x.join();
    for (int k = 0; k < 4; ++k)
      std::printf("#thread %d %016llx %016llx\n", k, (unsigned long long)serial[k], (unsigned long long)conc[k]);
  }
  if (only == "plancache") {  // one handle, 14 Hamiltonians in turn: device bytes after each call
    qf_state* st = make(16, QF_C128);
    std::vector<qf_term> T(T16);
    for (int k = 0; k < 14; ++k) {
      T[0].coeff = T16[0].coeff + 1e-3 * (k + 1);  // a different term list each call
      const qf_status s = qf_energy_grad(st, 255, A16.data(), A16.size(), t16.data(), t16.size(), T.data(),
                                         T.size(), &e, g.data());
      std::printf("#plancache %d %d %zu\n", k, (int)s, stub::live_bytes());
    }
    qf_state_destroy(st);
    std::printf("#plancache_after_destroy %zu\n", stub::live_bytes());
  }
  if (only == "sweep8") {  // an 8-qubit dUCCSD circuit on its sector state: the full-layout sector sweep
    const auto R = load<qf_rot>("rot8.bin");
    qf_state* st = make(8, QF_C128);
    qf_set_basis(st, 15);
    stub::reset();
    report("apply_circuit.8q.ucc", qf_apply_circuit(st, R.data(), R.size()));
    qf_state_destroy(st);
  }
  if (only == "multi8") {  // four parameter vectors of one 8-qubit system in one grouped call
    qf_state* st = make(8, QF_C128);
    report("energy_grad_multi.8q.c128", qf_energy_grad_multi(st, 15, A8.data(), A8.size(), t8.data(),
                                                             t8.size() / 4, 4, T8.data(), T8.size(), es.data(),
                                                             g.data()));
    qf_state_destroy(st);
  }
  if (only == "hpsi8") {  // a generic ansatz on 8 qubits: the gather H|psi> kernel and its tables
    const auto A = load<qf_arot>("ansatz_h8.bin");
    const auto t = load<double>("t_h8.bin");
    const auto H = load<qf_term>("ham8.bin");
    qf_state* st = make(8, QF_C128);
    report("energy_grad.8q.generic", qf_energy_grad(st, 0x35, A.data(), A.size(), t.data(), t.size(), H.data(),
                                                    H.size(), &e, g.data()));
    qf_state_destroy(st);
  }
  if (only.empty() || only == "general10") {
    qf_state* st = make(10, QF_C128);
    report("energy_grad.10q.general", qf_energy_grad(st, 31, A10.data(), A10.size(), t10.data(), t10.size(),
                                                     T10.data(), T10.size(), &e, g.data()));
    qf_state_destroy(st);
  }
  if (only.empty()) {
    for (int d = 0; d < 2; ++d) {
      const qf_dtype dt = d ? QF_C64 : QF_C128;
      const std::string sfx = d ? ".c64" : ".c128";
      qf_state* st = make(10, dt);
      qf_set_basis(st, 0x155);
      stub::reset();
      report("apply_circuit.10q.random" + sfx, qf_apply_circuit(st, R10.data(), R10.size()));
      report("expectation.10q.random" + sfx, qf_expectation(st, H10.data(), H10.size(), &re, &im));
      report("trotter.10q.random" + sfx, qf_trotter(st, H10.data(), H10.size(), 0.25, 2));
      qf_state_destroy(st);
      st = make(8, dt);
      report("energy_grad_multi.8q" + sfx,
             qf_energy_grad_multi(st, 15, A8.data(), A8.size(), t8.data(), t8.size() / 4, 4, T8.data(), T8.size(),
                                  es.data(), g.data()));
      qf_state_destroy(st);
    }
  }
  std::printf("#live_at_exit %zu\n", stub::live_bytes());  // every handle destroyed: nothing left
  return 0;
}
