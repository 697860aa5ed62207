"""The C ABI's host planning, run without a GPU.

qf_api.cu is compiled with g++ against a test double of the CUDA runtime and of
the kernel launchers (tests/hostplan/cuda_stub.cpp): device memory is host
memory, no kernel runs, and everything a call would send to the device (uploads
and the plain-data launch arguments) is hashed.  This covers the planner -- X-mask
grouping and its tables, the direct sector tables, block composites, the
part-local run plan, grouped small requests -- on every ABI path, and checks:
  * every path plans without error, and destroying the handles releases every
    device allocation; the plan cache stays bounded; handles planned from
    several host threads at once do not interfere;
  * plans are deterministic, and every plan rebuilt after qf_state_clear_plans
    sends the device the same bytes;
  * a call with new angles on a kept plan uploads only the new composites;
  * the part-local sweep plan of the 24-qubit dUCCSD evaluation moves exactly
    one item per (sector determinant, excitation) pair the excitation acts on;
  * each fused block's composite (Eq. 19's excitation factors, applied as one
    2^u x 2^u block on its active rows) and generator equal the dense products
    of its rotations computed by the oracle, and so do the grouped small
    requests' per-request block records and the sector sweep's blocks;
  * the X-mask groups' sign-pattern tables, and the direct sector tables of a
    molecular Hamiltonian, reproduce the oracle's Hamiltonian matrix elements;
  * the launches qf_apply_circuit and qf_trotter plan, replayed on a dense
    vector, give the oracle's state.
"""
import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HERE = os.path.join(ROOT, "tests", "hostplan")
CUDA_INC = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "include")


def _have_toolchain():
    return shutil.which("g++") is not None and os.path.exists(os.path.join(CUDA_INC, "cuda_runtime.h"))


@pytest.fixture(scope="module")
def suite(tmp_path_factory):
    if not _have_toolchain():
        pytest.skip("needs g++ and the CUDA headers")
    d = tmp_path_factory.mktemp("hostplan")
    exe = str(d / "plan_suite")
    inc = ["-I", os.path.join(ROOT, "include"), "-I", os.path.join(ROOT, "paper_2108_04413_gb300", "csrc"),
           "-I", CUDA_INC]
    cmd = (["g++", "-O1", "-std=c++17", "-w"] + inc +
           ["-x", "c++", os.path.join(ROOT, "paper_2108_04413_gb300", "csrc", "qf_api.cu"), "-x", "none",
            os.path.join(HERE, "cuda_stub.cpp"), os.path.join(HERE, "plan_suite.cpp"), "-o", exe, "-lpthread"])
    subprocess.run(cmd, check=True, capture_output=True, timeout=600)
    _write_inputs(str(d))
    return exe, str(d)


def _write_inputs(d):
    from paper_2108_04413_gb300 import prep
    from paper_2108_04413_gb300.abi import AROT_DTYPE
    from workloads import amplitudes, integrals

    def save(name, a):
        np.ascontiguousarray(a).tofile(os.path.join(d, name))

    # 16 qubits, half filling: the compact sector path
    h, g = integrals(8, 1)
    T16 = prep.molecular_hamiltonian(h, g)
    A16, ex16 = prep.uccsd_ansatz(8, 8)
    t16 = amplitudes(len(ex16), 1, 0.1)
    pool = A16.copy()
    pool["param"] = len(ex16) - 1 - A16["param"]
    idx, _ = prep.excited_determinants(ex16, 255)
    save("terms16.bin", T16), save("ansatz16.bin", A16), save("t16.bin", np.asarray(t16, np.float64))
    save("rot16.bin", prep.bind_thetas(A16, t16)), save("pool16.bin", pool)
    save("dets16.bin", np.asarray(idx, np.uint64))
    # 10 qubits: a particle-number-changing rotation first, so the dUCCSD factors
    # that follow run as general sparse blocks (their composites are checked)
    h, g = integrals(5, 3)
    A, ex10 = prep.uccsd_ansatz(5, 5)
    A10 = np.zeros(len(A) + 1, dtype=AROT_DTYPE)
    A10[0] = (1, 0, 1.0, 0, 0)
    A10[1:] = A
    A10["param"][1:] += 1
    save("ansatz10.bin", A10), save("t10.bin", amplitudes(len(ex10) + 1, 5, 0.2))
    save("terms10.bin", prep.molecular_hamiltonian(h, g))
    save("rot10.bin", prep.random_circuit(10, 200, 7)), save("ham10.bin", prep.random_hamiltonian(10, 300, 9))
    # 8 qubits, four parameter vectors in one grouped call
    h, g = integrals(4, 0)
    A8, ex8 = prep.uccsd_ansatz(4, 4)
    save("ansatz8.bin", A8), save("terms8.bin", prep.molecular_hamiltonian(h, g))
    save("t8.bin", np.stack([amplitudes(len(ex8), 20 + k, 0.15) for k in range(4)]).astype(np.float64))


def _run(suite, *args, env=None):
    exe, d = suite
    out = subprocess.run([exe, d, *args], check=True, capture_output=True, text=True, timeout=600,
                         env=dict(os.environ, **(env or {}))).stdout
    assert "#error" not in out, out
    rows = {}
    for line in out.splitlines():
        if line.startswith("#live_at_exit"):
            assert int(line.split()[1]) == 0, "device memory left after every handle was destroyed"
            continue
        name, status, copies, h2d, digest = line.split()
        rows[name] = (int(status), int(copies), int(h2d), digest)
    return rows


def test_every_abi_path_plans_on_the_host(suite):
    rows = _run(suite)
    assert len(rows) == 17
    for name, (status, copies, _, _) in rows.items():
        assert status == 0, name
        assert copies > 0, name
    assert rows["energy_grad.16q.cold"][2] > 0 and rows["energy_grad.10q.general"][2] > 0


def test_plans_are_deterministic_and_rebuilt_identically(suite):
    a, b = _run(suite), _run(suite)
    assert a == b
    assert a["energy_grad.16q.rebuilt"] == a["energy_grad.16q.rebuilt_again"]


def test_new_angles_upload_only_the_composites(suite):
    rows = _run(suite, "sector16")
    cold, warm = rows["energy_grad.16q.rebuilt_again"], rows["energy_grad.16q.warm"]
    assert 0 < warm[2] < cold[2] / 2
    assert warm[3] != cold[3]


def _sparse_args(raw, layout):
    size, o_u, o_nr, o_ncls, o_nzc, o_supp, o_pat, o_zc, o_m, o_q, max_supp, max_rows, max_cls = layout
    assert len(raw) % size == 0
    out = []
    for k in range(len(raw) // size):
        b = raw[k * size:(k + 1) * size]
        i32 = lambda off, cnt=1: np.frombuffer(b, np.int32, cnt, off)  # noqa: E731
        u, nr, ncls, nzc = (int(i32(o)[0]) for o in (o_u, o_nr, o_ncls, o_nzc))
        cmat = np.frombuffer(b, np.float64, 2 * max_cls * max_rows * max_rows, o_m).view(np.complex128)
        qmat = np.frombuffer(b, np.float64, 2 * max_cls * max_rows * max_rows, o_q).view(np.complex128)
        out.append(dict(u=u, nr=nr, ncls=ncls, nzc=nzc, supp=i32(o_supp, u).tolist(),
                        pat=np.frombuffer(b, np.uint64, nr, o_pat).tolist(),
                        zc=np.frombuffer(b, np.uint64, nzc, o_zc).tolist(),
                        M=cmat.reshape(max_cls, max_rows, max_rows)[:ncls, :nr, :nr],
                        Q=qmat.reshape(max_cls, max_rows, max_rows)[:ncls, :nr, :nr]))
    return out


def test_sparse_composites_match_dense_products(suite, tmp_path):
    """Every fused dUCCSD factor of the general path: M + I on the active rows is
    the product of the factor's rotations (adjoint sweep: its inverse), and Q is
    sum_k coeff_k P_k, for every sign class of the Z strings outside the support;
    rows outside the active set are left unchanged."""
    from oracle import pauli
    from paper_2108_04413_gb300.abi import AROT_DTYPE

    exe, d = suite
    layout = [int(v) for v in subprocess.run([exe, d, "layout"], check=True, capture_output=True,
                                             text=True).stdout.split()]
    _run(suite, "general10", env={"QF_STUB_DUMP_DIR": str(tmp_path)})
    n = 10
    A = np.fromfile(os.path.join(d, "ansatz10.bin"), dtype=AROT_DTYPE)
    t = np.fromfile(os.path.join(d, "t10.bin"), dtype=np.float64)
    runs = {}
    for x, z, c, p in zip(A["x"].tolist(), A["z"].tolist(), A["coeff"].tolist(), A["param"].tolist()):
        runs.setdefault(int(x), []).append((int(z), float(c), int(p)))
    fwd = _sparse_args((tmp_path / "fwd.bin").read_bytes(), layout)
    adj = _sparse_args((tmp_path / "adj.bin").read_bytes(), layout)
    assert len(fwd) == len(runs) - 1 == len(adj)  # every factor but the single X rotation
    assert {a["ncls"] for a in fwd} == {1, 2}  # factors with and without Z strings outside the support
    for blocks, inverse in ((fwd, False), (adj, True)):
        for a in blocks:
            x = sum(1 << q for q in a["supp"])
            rots = [(x, z, c * t[p]) for z, c, p in runs[x]]
            assert 0 <= a["nzc"] <= 2 and a["ncls"] == 1 << a["nzc"]
            for cls in range(a["ncls"]):
                # a basis state off the support whose outside-Z parities give this class
                b0 = next(b for b in range(1 << n) if not (b & x) and all(
                    (bin(zc & b).count("1") & 1) == ((cls >> j) & 1) for j, zc in enumerate(a["zc"])))
                rows = [b0 ^ p for p in a["pat"]]
                for j, rj in enumerate(rows):
                    col = pauli.apply_rotations(pauli.basis_state(n, rj), n, rots)
                    gen = sum(c * pauli.apply(pauli.basis_state(n, rj), n, x, z) for z, c, _ in runs[x])
                    assert abs(np.linalg.norm(col[rows]) - 1.0) < 1e-13  # no amplitude leaves the active rows
                    for i, ri in enumerate(rows):
                        u = np.conj(pauli.apply_rotations(pauli.basis_state(n, ri), n, rots)[rj]) if inverse \
                            else col[ri]
                        assert abs(a["M"][cls, i, j] + (i == j) - u) < 1e-13
                        assert abs(a["Q"][cls, i, j] - gen[ri]) < 1e-13
                # a support pattern outside the active set is left unchanged
                rest = [r for r in range(1 << a["u"]) if sum(((r >> k) & 1) << q for k, q in
                                                             enumerate(a["supp"])) not in a["pat"]]
                if rest:
                    r0 = b0 ^ sum(((rest[0] >> k) & 1) << q for k, q in enumerate(a["supp"]))
                    col = pauli.apply_rotations(pauli.basis_state(n, r0), n, rots)
                    assert abs(col[r0] - 1.0) < 1e-13


def test_sweep_plan_items_at_24_qubits_count_the_sector_pairs(suite):
    """The 24-qubit dUCCSD evaluation's run plan: its per-run items (the units the
    sweeps' flops and log traffic are counted in) add up to the brute-force count
    of (sector determinant, excitation) pairs with the excitation's occupied
    orbitals filled and its virtual orbitals empty."""
    from oracle import sector
    from paper_2108_04413_gb300 import prep
    from workloads import WORKLOADS, amplitudes, integrals

    exe, d = suite
    cfg = WORKLOADS["ucc24"]
    h, g = integrals(cfg["n_orb"], cfg["seed"])
    A, exs = prep.uccsd_ansatz(cfg["n_orb"], cfg["n_el"])
    prep.molecular_hamiltonian(h, g).tofile(os.path.join(d, "terms_ri.bin"))
    A.tofile(os.path.join(d, "ansatz_ri.bin"))
    amplitudes(len(exs), cfg["seed"], cfg["t_sigma"]).astype(np.float64).tofile(os.path.join(d, "t_ri.bin"))
    det = (1 << cfg["n_el"]) - 1
    out = subprocess.run([exe, d, "runitems", str(cfg["n_qubits"]), str(det)], check=True, capture_output=True,
                         text=True, timeout=600).stdout
    items = np.array([int(v) for v in out.split()], dtype=np.int64)
    na, nb = sector.counts_of(det)
    dets = sector.sector_dets(cfg["n_orb"], na, nb)
    expect = 0
    for occ, vir in exs:
        om = np.uint64(sum(1 << q for q in occ))
        vm = np.uint64(sum(1 << q for q in vir))
        expect += int(np.count_nonzero(((dets & om) == om) & ((dets & vm) == 0)))
    assert len(exs) == 1818 and len(dets) == 853776
    assert len(items) > 1 and (items > 0).all()
    assert int(items.sum()) == expect == 128172240
    # the committed DRAM captures of the sweeps are scaled by these runs' items:
    # they must be the runs the captures measured
    import json

    traffic = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))
    for key in ("k_sector_run (forward)", "k_sector_run (reverse)"):
        rec = traffic[key]
        assert rec["n_runs"] == len(items)
        assert sum(int(items[r]) for r in rec["runs"]) == rec["items"], key


def test_xmask_group_tables_reproduce_the_hamiltonian(suite, tmp_path):
    """The X-mask grouping (Eq. 18 evaluated group by group): for every group x and
    every basis state b, the group's chunk tables read at b's sign patterns sum to
    <b XOR x| H |b>.  The Hamiltonian mixes a group whose Z masks span three
    dimensions (one chunk of combinations), a group spanning more than four (chunks
    of four terms), the diagonal group, odd-Y terms and repeated terms."""
    from oracle import pauli
    from paper_2108_04413_gb300.abi import as_arots, as_terms

    exe, d = suite
    n = 8
    rng = np.random.default_rng(18)
    basis = rng.integers(0, 1 << n, 3)
    span = [int(np.bitwise_xor.reduce(basis[[k for k in range(3) if (m >> k) & 1]], initial=0)) for m in range(8)]
    xs = [0b00110101] * 12 + [0b11000011] * 10 + [0] * 15 + list(rng.integers(0, 1 << n, 150))
    zs = [span[rng.integers(0, 8)] for _ in range(12)] + list(rng.integers(0, 1 << n, 10 + 15 + 150))
    zs[40], xs[40] = zs[41], xs[41]  # a repeated term
    T = as_terms(np.array(xs), np.array(zs), rng.normal(size=len(xs)))
    A = as_arots(rng.integers(0, 1 << n, 30), rng.integers(0, 1 << n, 30), rng.normal(size=30), rng.integers(0, 6, 30))
    T.tofile(os.path.join(d, "ham8.bin"))
    A.tofile(os.path.join(d, "ansatz_h8.bin"))
    rng.normal(size=6).tofile(os.path.join(d, "t_h8.bin"))
    _run(suite, "hpsi8", env={"QF_STUB_DUMP_DIR": str(tmp_path)})
    gsize, o_x, o_nchunk, o_chunk0, csize, o_z, o_tab, _, npat, kterms = (
        int(v) for v in subprocess.run([exe, d, "tables"], check=True, capture_output=True, text=True).stdout.split())
    graw, craw = (tmp_path / "groups.bin").read_bytes(), (tmp_path / "hchunks.bin").read_bytes()
    H = pauli.dense_sum(n, [(int(x), int(z), float(c)) for x, z, c in zip(T["x"], T["z"], T["coeff"])])
    seen = set()
    b = np.arange(1 << n, dtype=np.uint64)
    for k in range(len(graw) // gsize):
        g = graw[k * gsize:(k + 1) * gsize]
        x = int(np.frombuffer(g, np.uint64, 1, o_x)[0])
        nchunk, chunk0 = (int(np.frombuffer(g, np.int32, 1, o)[0]) for o in (o_nchunk, o_chunk0))
        seen.add(x)
        D = np.zeros(1 << n, dtype=complex)
        for c in range(chunk0, chunk0 + nchunk):
            ch = craw[c * csize:(c + 1) * csize]
            z = np.frombuffer(ch, np.uint64, kterms, o_z)
            tab = np.frombuffer(ch, np.float64, 2 * npat, o_tab).view(np.complex128)
            pat = sum(((pauli.popcount(z[j] & b) & 1).astype(np.int64) << j) for j in range(kterms))
            D += tab[pat]
        np.testing.assert_allclose(D, H[b.astype(np.int64) ^ x, b.astype(np.int64)], rtol=0, atol=1e-13)
    assert seen == {int(v) for v in T["x"]}
    assert len(seen) == len(graw) // gsize


def _direct_tables(raw):
    head = np.frombuffer(raw, np.int32, 4, 0)
    n, ne, no = (int(v) for v in head[:3])
    inv_fix = float(np.frombuffer(raw, np.float64, 1, 16)[0])
    pe, po = ne * (ne - 1) // 2, no * (no - 1) // 2
    sizes = [("wab", np.float64, ne * ne * no * no), ("waa", np.float64, max(1, pe * pe)),
             ("wbb", np.float64, max(1, po * po)), ("s1a", np.int64, ne * ne * (n + 1)),
             ("s1b", np.int64, no * no * (n + 1)), ("dg", np.int64, 1 + n + n * n)]
    off, t = 24, dict(n=n, ne=ne, no=no, inv_fix=inv_fix)
    for name, dt, cnt in sizes:
        t[name] = np.frombuffer(raw, dt, cnt, off)
        off += cnt * 8
    assert off == len(raw)
    return t


def _h_from_direct(t, c, c2):
    """<c|H|c2> as the direct tables state it: the diagonal K + sum U + sum V over
    c's occupied qubits; a single o -> v (c occupies o) A + sum of B over c's other
    occupied qubits; doubles one weight; each off-diagonal entry signed by the
    parities of c's occupied qubits below each moved qubit."""
    n, ne, no = t["n"], t["ne"], t["no"]
    occ = [q for q in range(n) if (c >> q) & 1]
    pp = lambda q: bin(c & ((1 << q) - 1)).count("1") & 1  # noqa: E731
    pr = lambda i, j: i + j * (j - 1) // 2  # noqa: E731
    d = c ^ c2
    gone = [q for q in range(n) if (d >> q) & 1 and (c >> q) & 1]   # occupied in c, empty in c2
    new = [q for q in range(n) if (d >> q) & 1 and (c2 >> q) & 1]
    if d == 0:
        dg = t["dg"]
        v = int(dg[0]) + sum(int(dg[1 + r]) for r in occ)
        v += sum(int(dg[1 + n + r * n + s]) for i, r in enumerate(occ) for s in occ[i + 1:])
        return v * t["inv_fix"]
    sign = (-1) ** (sum(pp(q) for q in gone + new) & 1)
    if len(gone) == 1:
        o, v = gone[0], new[0]
        if (o & 1) != (v & 1):
            return 0.0
        tab, m = (t["s1a"], ne) if o % 2 == 0 else (t["s1b"], no)
        row = tab[((o >> 1) * m + (v >> 1)) * (n + 1):][:n + 1]
        w = int(row[0]) + sum(int(row[1 + r]) for r in occ if r != o)
        return sign * w * t["inv_fix"]
    if len(gone) == 2:
        ga = [q >> 1 for q in gone if q % 2 == 0]
        na_ = [q >> 1 for q in new if q % 2 == 0]
        gb = [q >> 1 for q in gone if q % 2 == 1]
        nb_ = [q >> 1 for q in new if q % 2 == 1]
        if len(ga) != len(na_):
            return 0.0
        if len(ga) == 1:
            return sign * t["wab"][((ga[0] * ne + na_[0]) * no + gb[0]) * no + nb_[0]]
        if len(ga) == 2:
            return sign * t["waa"][pr(*ga) * (ne * (ne - 1) // 2) + pr(*na_)]
        return sign * t["wbb"][pr(*gb) * (no * (no - 1) // 2) + pr(*nb_)]
    return 0.0


@pytest.mark.parametrize("case", ["direct8", "direct10"])
def test_direct_sector_tables_reproduce_the_hamiltonian(suite, tmp_path, case):
    """The direct sector tables of a molecular Hamiltonian (Eq. 1 through the
    Jordan-Wigner map of Eq. 15-16): every matrix element between two determinants
    of the sector, as the tables state it, equals the oracle's dense Hamiltonian
    (half filling at 8 qubits; 3 alpha and 2 beta electrons at 10)."""
    from oracle import pauli, sector
    from paper_2108_04413_gb300.abi import TERM_DTYPE

    exe, d = suite
    _run(suite, case, env={"QF_STUB_DUMP_DIR": str(tmp_path)})
    t = _direct_tables((tmp_path / "direct.bin").read_bytes())
    n = t["n"]
    T = np.fromfile(os.path.join(d, "terms8.bin" if case == "direct8" else "terms10.bin"), dtype=TERM_DTYPE)
    H = pauli.dense_sum(n, [(int(x), int(z), float(c)) for x, z, c in zip(T["x"], T["z"], T["coeff"])])
    assert np.abs(H.imag).max() == 0.0
    na, nb = sector.counts_of(15 if case == "direct8" else 31)
    dets = [int(v) for v in sector.sector_dets(n // 2, na, nb)]
    got = np.array([[_h_from_direct(t, c, c2) for c2 in dets] for c in dets])
    want = H.real[np.ix_(dets, dets)]
    assert np.abs(want).max() > 0.1
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-12)


def test_grouped_request_records_match_dense_products(suite, tmp_path):
    """qf_energy_grad_multi's per-request block records (one CTA per request):
    for every request and dUCCSD factor, the forward composite minus identity on
    the factor's two active determinants, its inverse, and the generator's
    coupling q01 (Q = i Qi), per sign class of the Z strings outside the support,
    equal the oracle's dense products of the factor's rotations at that request's
    angles."""
    from oracle import pauli
    from paper_2108_04413_gb300.abi import AROT_DTYPE

    exe, d = suite
    _run(suite, "multi8", env={"QF_STUB_DUMP_DIR": str(tmp_path)})
    bsize, o_pat, o_zc, o_nzc, ncoef, _ = (
        int(v) for v in subprocess.run([exe, d, "secblk"], check=True, capture_output=True, text=True).stdout.split())
    braw = (tmp_path / "small_blks.bin").read_bytes()
    coef = np.frombuffer((tmp_path / "small_coef.bin").read_bytes(), np.float64)
    A = np.fromfile(os.path.join(d, "ansatz8.bin"), dtype=AROT_DTYPE)
    rows_t = np.fromfile(os.path.join(d, "t8.bin"), dtype=np.float64).reshape(4, -1)
    n, nblk = 8, len(braw) // bsize
    # a fresh handle plans with the first request (a single evaluation), then
    # groups the rest in one launch
    nreq = coef.size // (nblk * ncoef)
    assert nblk == rows_t.shape[1] and coef.size == nreq * nblk * ncoef and nreq == 3
    coef = coef.reshape(nreq, nblk, ncoef)
    rows_t = rows_t[4 - nreq:]
    runs = {}
    for x, z, c, p in zip(A["x"].tolist(), A["z"].tolist(), A["coeff"].tolist(), A["param"].tolist()):
        runs.setdefault(int(x), []).append((int(z), float(c), int(p)))
    for b in range(nblk):
        raw = braw[b * bsize:(b + 1) * bsize]
        pat = [int(v) for v in np.frombuffer(raw, np.uint64, 2, o_pat)]
        nzc = int(np.frombuffer(raw, np.int32, 1, o_nzc)[0])
        zc = [int(v) for v in np.frombuffer(raw, np.uint64, nzc, o_zc)]
        x = pat[0] ^ pat[1]
        for k in range(nreq):
            rots = [(x, z, c * rows_t[k, p]) for z, c, p in runs[x]]
            v = coef[k, b]
            for cls in range(1 << nzc):
                b0 = next(s for s in range(1 << n) if not (s & x) and all(
                    (bin(m & s).count("1") & 1) == ((cls >> j) & 1) for j, m in enumerate(zc)))
                dets = [b0 ^ p for p in pat]
                U = np.array([[pauli.apply_rotations(pauli.basis_state(n, cj), n, rots)[ci] for cj in dets]
                              for ci in dets])
                Q = np.array([[sum(c * pauli.apply(pauli.basis_state(n, cj), n, x, z)[ci] for z, c, _ in runs[x])
                               for cj in dets] for ci in dets])
                assert np.abs(U.imag).max() < 1e-15
                np.testing.assert_allclose(v[4 * cls:4 * cls + 4].reshape(2, 2), U.real - np.eye(2), atol=1e-13)
                np.testing.assert_allclose(v[16 + 4 * cls:20 + 4 * cls].reshape(2, 2), U.real.T - np.eye(2),
                                           atol=1e-13)
                assert abs(v[32 + cls] - (Q[0, 1] / 1j)) < 1e-13


def test_sector_sweep_blocks_match_dense_products(suite, tmp_path):
    """qf_apply_circuit of an 8-qubit dUCCSD circuit on its sector state runs the
    full-layout sector sweep: every block's real composite minus identity on its
    two active determinants, per sign class of the Z strings outside the support,
    equals the oracle's dense product of the excitation's rotations."""
    from oracle import pauli
    from paper_2108_04413_gb300 import prep
    from paper_2108_04413_gb300.abi import AROT_DTYPE

    exe, d = suite
    A = np.fromfile(os.path.join(d, "ansatz8.bin"), dtype=AROT_DTYPE)
    t = np.fromfile(os.path.join(d, "t8.bin"), dtype=np.float64).reshape(4, -1)[0]
    R = prep.bind_thetas(A, t)
    R.tofile(os.path.join(d, "rot8.bin"))
    _run(suite, "sweep8", env={"QF_STUB_DUMP_DIR": str(tmp_path)})
    bsize, o_pat, o_zc, o_nzc, _, o_m = (
        int(v) for v in subprocess.run([exe, d, "secblk"], check=True, capture_output=True, text=True).stdout.split())
    braw = (tmp_path / "sweep_blks.bin").read_bytes()
    runs = {}
    for x, z, th in zip(R["x"].tolist(), R["z"].tolist(), R["theta"].tolist()):
        runs.setdefault(int(x), []).append((int(x), int(z), float(th)))
    n, nblk = 8, len(braw) // bsize
    assert nblk == len(runs) == t.size
    for b in range(nblk):
        raw = braw[b * bsize:(b + 1) * bsize]
        pat = [int(v) for v in np.frombuffer(raw, np.uint64, 2, o_pat)]
        nzc = int(np.frombuffer(raw, np.int32, 1, o_nzc)[0])
        zc = [int(v) for v in np.frombuffer(raw, np.uint64, nzc, o_zc)]
        m = np.frombuffer(raw, np.float64, 16, o_m).reshape(4, 2, 2)
        rots = runs[pat[0] ^ pat[1]]
        for cls in range(1 << nzc):
            b0 = next(s for s in range(1 << n) if not (s & (pat[0] ^ pat[1])) and all(
                (bin(mz & s).count("1") & 1) == ((cls >> j) & 1) for j, mz in enumerate(zc)))
            dets = [b0 ^ p for p in pat]
            U = np.array([[pauli.apply_rotations(pauli.basis_state(n, cj), n, rots)[ci] for cj in dets]
                          for ci in dets])
            assert np.abs(U.imag).max() < 1e-15
            np.testing.assert_allclose(m[cls], U.real - np.eye(2), atol=1e-13)


@pytest.mark.parametrize("n", [10, 12, 14, 16, 18])
def test_serving_footprint_bounds_the_handle_memory(suite, n):
    """Serving admits a system by serving.footprint_bytes: it must bound the
    device bytes a handle really holds after an evaluation (the state, the
    compact sector copy, the forward log, item maps, run descriptors, plan
    tables and work buffers), without overstating them more than 2.5 times."""
    from paper_2108_04413_gb300 import prep
    from paper_2108_04413_gb300.serving import footprint_bytes
    from workloads import amplitudes, integrals

    exe, d = suite
    h, g = integrals(n // 2, 100 + n)
    T = prep.molecular_hamiltonian(h, g)
    A, exs = prep.uccsd_ansatz(n // 2, n // 2)
    T.tofile(os.path.join(d, "terms_fp.bin"))
    A.tofile(os.path.join(d, "ansatz_fp.bin"))
    np.asarray(amplitudes(len(exs), n, 0.1), np.float64).tofile(os.path.join(d, "t_fp.bin"))
    det = (1 << (n // 2)) - 1
    for dtype in ("c128", "c64"):
        out = subprocess.run([exe, d, "footprint", str(n), dtype, str(det)], check=True, capture_output=True,
                             text=True, timeout=600).stdout
        assert "#error" not in out, out
        held = int(out.split()[0])
        bound = footprint_bytes(n, dtype, det, A, len(T))
        assert held <= bound <= 2.5 * held, (n, dtype, held, bound)


def test_plan_cache_is_bounded_and_released(suite):
    """A handle that receives new Hamiltonians keeps at most a fixed number of
    plans (least recently used evicted with their device tables): its device
    bytes stop growing, and destroying it releases everything."""
    exe, d = suite
    out = subprocess.run([exe, d, "plancache"], check=True, capture_output=True, text=True, timeout=600).stdout
    rows = [line.split() for line in out.splitlines() if line.startswith("#plancache ")]
    assert [int(r[2]) for r in rows] == [0] * 14
    held = [int(r[3]) for r in rows]
    assert held[1] > held[0]  # a second plan is kept
    assert max(held[8:]) == held[8] == held[-1]  # from the ninth on, each new plan replaces the oldest
    assert int(out.split("#plancache_after_destroy")[1].split()[0]) == 0


def test_rejected_calls_leave_the_handle_working(suite):
    """Invalid inputs (a Pauli letter past the register, a parameter index past
    the vector, a non-finite angle, a determinant past the register, a NULL
    array) are rejected with QF_EINVAL before anything is planned or sent; the
    handle then evaluates normally and holds what a fresh handle would."""
    exe, d = suite
    out = subprocess.run([exe, d, "errors"], check=True, capture_output=True, text=True, timeout=600).stdout
    status = {l.split()[1]: int(l.split()[2]) for l in out.splitlines() if l.startswith("#status")}
    QF_OK, QF_EINVAL = 0, 1
    assert status == {"mask": QF_EINVAL, "param": QF_EINVAL, "angle": QF_EINVAL, "det": QF_EINVAL,
                      "null": QF_EINVAL, "valid": QF_OK}
    clean, held = (int(v) for v in out.split("#held")[1].split()[:2])
    assert held == clean


def test_handles_plan_independently_on_concurrent_threads(suite):
    """Serving evaluates several handles from several host threads at once (the
    planner's worker pool is shared): four handles planned and evaluated
    concurrently send the device exactly what each sends alone."""
    exe, d = suite
    out = subprocess.run([exe, d, "threads"], check=True, capture_output=True, text=True, timeout=600).stdout
    assert "#error" not in out, out
    rows = [line.split() for line in out.splitlines() if line.startswith("#thread")]
    assert len(rows) == 4
    assert all(r[2] == r[3] for r in rows)
    assert len({r[2] for r in rows}) == 4  # different angles, different uploads


def test_28_qubit_workload_plans_deterministically(suite):
    """The largest workload: 500 random Pauli exponentials and the 20000-term sum
    on a 28-qubit register (4 GiB of complex128) plan without error, the same way
    twice, and release their memory."""
    from paper_2108_04413_gb300 import prep
    from workloads import WORKLOADS

    exe, d = suite
    seed = WORKLOADS["sweep28"]["seed"]
    prep.random_circuit(28, 500, seed).tofile(os.path.join(d, "rot28.bin"))
    prep.random_hamiltonian(28, 20000, seed).tofile(os.path.join(d, "ham28.bin"))
    a, b = _run(suite, "big28"), _run(suite, "big28")
    assert a == b and len(a) == 4
    for name, (status, copies, _, _) in a.items():
        assert status == 0 and copies > 0, name
    assert a["expectation.28q.c128"][2] > 0


def _replay(raw, n, sparse_layout, secblk_layout):
    """The dense state the logged launches produce (the stored values; the kept
    scale is applied by the caller).  A rotation record applies A*I - i*B*P with
    P|b> = i^popc(x&z) (-1)^popc(z&b) |b^x> (the oracle's convention)."""
    from oracle import pauli

    ssize, o_u, o_nr, o_ncls, o_nzc, o_supp, o_pat, o_zc, o_m, _, _, max_rows, max_cls = sparse_layout
    bsize, b_pat, b_zc, b_nzc, _, b_m = secblk_layout
    psi = None
    off, nops = 0, 0
    b = np.arange(1 << n, dtype=np.int64)

    def take(dt, cnt=1):
        nonlocal off
        v = np.frombuffer(raw, dt, cnt, off)
        off += v.nbytes
        return v

    def rot(x, z, A, B):
        return A * psi - 1j * B * pauli.apply(psi, n, x, z)

    def block(x, pat, zc, mats):  # (M_c + I) on the active rows of every outside configuration
        out = psi.copy()
        for s0 in range(1 << n):
            if s0 & x:
                continue
            cls = sum(((bin(zc[j] & s0).count("1") & 1) << j) for j in range(len(zc)))
            rows = [s0 | p for p in pat]
            out[rows] = psi[rows] + mats[cls] @ psi[rows]
        return out

    while off < len(raw):
        kind = int(take(np.int32)[0])
        nops += 1
        if kind == 1:
            psi = pauli.basis_state(n, int(take(np.uint64)[0]))
        elif kind == 2:
            x, z = (int(v) for v in take(np.uint64, 2))
            A, B = take(np.float64, 2)
            psi = rot(x, z, A, B)
        elif kind == 3:
            m, s = (int(v) for v in take(np.int32, 2))
            sbits = [int(v) for v in take(np.int32, s)]
            expand = lambda v: sum(1 << sbits[q] for q in range(s) if (v >> q) & 1)  # noqa: E731
            for _ in range(m):
                xl, zl = (int(v) for v in take(np.uint32, 2))
                zout = int(take(np.uint64)[0])
                A, B = take(np.float64, 2)
                psi = rot(expand(xl), expand(zl) | zout, A, B)
        elif kind == 4:
            a = _sparse_args(raw[off:off + ssize], sparse_layout)[0]
            off += ssize
            psi = block(sum(1 << q for q in a["supp"]), a["pat"], a["zc"], a["M"])
        elif kind == 5:
            nblk = int(take(np.int32)[0])
            for _ in range(nblk):
                rec = raw[off:off + bsize]
                off += bsize
                pat = [int(v) for v in np.frombuffer(rec, np.uint64, 2, b_pat)]
                nzc = int(np.frombuffer(rec, np.int32, 1, b_nzc)[0])
                zc = [int(v) for v in np.frombuffer(rec, np.uint64, nzc, b_zc)]
                mats = np.frombuffer(rec, np.float64, 16, b_m).reshape(4, 2, 2)
                psi = block(pat[0] ^ pat[1], pat, zc, mats)
        elif kind == 6:
            psi = psi * float(take(np.float64)[0])
        else:
            raise AssertionError(f"unknown op {kind}")
    return psi, nops


def _layouts(exe, d):
    run = lambda mode: [int(v) for v in subprocess.run([exe, d, mode], check=True, capture_output=True,  # noqa: E731
                                                        text=True).stdout.split()]
    return run("layout"), run("secblk")


@pytest.mark.parametrize("case", ["random13", "ucc10_general", "ucc8_sector", "trotter10"])
def test_circuit_plans_replay_to_the_oracle_state(suite, tmp_path, case):
    """qf_apply_circuit and qf_trotter as planned: the launches they would make
    (unfused rotations, fused tiles with their tile-local bit maps, sparse blocks,
    sector sweeps) and the scale the state keeps aside, replayed on a dense
    vector, give the oracle's state.  Cases: random weight-2..8 exponentials on 13
    qubits (tile fusion, diagonal and single-flip rotations); a dUCCSD circuit on
    10 qubits after a particle-number-changing rotation (general sparse blocks);
    a dUCCSD circuit on its 8-qubit sector state (one sector sweep); a first-order
    Trotter evolution of a random Hamiltonian on 10 qubits."""
    from oracle import pauli
    from paper_2108_04413_gb300 import prep
    from paper_2108_04413_gb300.abi import AROT_DTYPE, ROT_DTYPE, TERM_DTYPE
    from workloads import amplitudes

    exe, d = suite
    extra = []
    if case == "random13":
        n, det = 13, 0b1010110100101
        R = prep.random_circuit(n, 150, 13)
    elif case == "ucc10_general":
        n, det = 10, 31
        A10 = np.fromfile(os.path.join(d, "ansatz10.bin"), dtype=AROT_DTYPE)
        t10 = np.fromfile(os.path.join(d, "t10.bin"), dtype=np.float64)
        R = prep.bind_thetas(A10, t10)
    elif case == "ucc8_sector":
        n, det = 8, 15
        A8, ex8 = prep.uccsd_ansatz(4, 4)
        R = prep.bind_thetas(A8, amplitudes(len(ex8), 3, 0.3))
    else:
        n, det = 10, 0b0101010101
        T = prep.random_hamiltonian(n, 40, 21)
        T.tofile(os.path.join(d, "terms_c.bin"))
        extra = ["trotter"]
        R = np.zeros(0, dtype=ROT_DTYPE)
        for _ in range(3):  # the oracle's own Trotter steps, written out as rotations
            R = np.concatenate([R, np.array([(x, z, c * 0.3 / 3) for x, z, c in zip(T["x"], T["z"], T["coeff"])],
                                            dtype=ROT_DTYPE)])
        assert T.dtype == TERM_DTYPE
    R.tofile(os.path.join(d, "rot_c.bin"))
    sl, bl = _layouts(exe, d)
    for dtype in ("c128", "c64"):
        dump = tmp_path / dtype
        dump.mkdir()
        out = subprocess.run([exe, d, "circuit", str(n), str(det), dtype, *extra], check=True, capture_output=True,
                             text=True, timeout=600, env=dict(os.environ, QF_STUB_DUMP_DIR=str(dump))).stdout.split()
        assert int(out[0]) == 0
        psi, nops = _replay((dump / "ops.bin").read_bytes(), n, sl, bl)
        psi = psi * float(out[1])
        ref = pauli.apply_rotations(pauli.basis_state(n, det), n, [(int(x), int(z), float(t)) for x, z, t in
                                                                    zip(R["x"], R["z"], R["theta"])])
        assert nops >= 2
        np.testing.assert_allclose(psi, ref, rtol=0, atol=1e-11)
