"""Host-logic checks of the library's symbolic analysis (csrc/ddlr_plan.cpp),
on the CPU: tests/plan_probe.cpp calls build_plan on a pattern and writes the
plan's arrays, and every property is checked here against its definition,
computed independently with numpy:

* Sec. 2.1 classification: a node is an interface node iff it has a
  neighbour in another subdomain; block b < p holds exactly the interior
  nodes of subdomain b, block p the interface nodes; iface_rank ranks the
  interface nodes by original index;
* factor pattern (eq. split and the local solvers of Sec. 5): for IC(0) the
  strictly lower entries of a block are its graph's edges (A restricted to
  the block, plus the pattern of Ehat Ehat^T for interior blocks; the
  Chebyshev mode keeps the couplings of C_a inside one subdomain, the
  approximate inverse none), each once, in the row of the endpoint
  eliminated later; natural order eliminates by ascending original index,
  multicolour order of a bipartite graph puts the colour class of each
  component's lowest node first; exact mode: the fill pattern of a dense
  Cholesky factor of the block; value sources (A's entries, the Ehat Ehat^T
  products, the a^2 of C_a's diagonal);
* levels: 1 + the largest level of a row's lower columns; rows sorted by
  level inside each block; two levels for multicolour grids;
* the schedule is the stable sort of the rows by level; the level-order
  descriptors list the same rows with their slots; the chunk tables cover
  every row exactly once in chunks of at most 256 rows of one level record;
* the sliced-ELL solve layouts hold each row's L entries and its L^T entries
  (ascending row), padding slots pointing at rows final before use;
  map_l / map_u give every entry's slot;
* Ehat, Ehat^T and the SpMV layout hold A's entries in device order.
"""
import os
import shutil
import subprocess

import numpy as np
import pytest

import workloads as W

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(ROOT, "paper_1505_04341_gb300", "csrc")


@pytest.fixture(scope="module")
def probe():
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    out_dir = os.path.join(HERE, "_build")
    os.makedirs(out_dir, exist_ok=True)
    exe = os.path.join(out_dir, "plan_probe")
    srcs = [os.path.join(HERE, "plan_probe.cpp"), os.path.join(CSRC, "ddlr_plan.cpp")]
    if not os.path.exists(exe) or os.path.getmtime(exe) < max(
            os.path.getmtime(s) for s in srcs + [os.path.join(CSRC, "ddlr_plan.h")]):
        tmp = exe + f".{os.getpid()}.tmp"
        subprocess.check_call([gxx, "-O2", "-std=c++17", "-pthread", "-I" + os.path.join(ROOT, "include"),
                               "-I" + CSRC, "-o", tmp] + srcs)
        os.replace(tmp, exe)
    return exe


def run_plan(probe, A, part, p, tag, variant=1, k=2, factor=0, c_order=0, b_order=0, c_solver=0, fill_level=0):
    n, rp, ci, va = A
    d = os.path.join(HERE, "_build")
    fin, fout = os.path.join(d, f"plan_in_{tag}.bin"), os.path.join(d, f"plan_out_{tag}.bin")
    with open(fin, "wb") as f:
        np.array([n, len(ci), p, variant, k, factor, c_order, b_order, c_solver, fill_level], np.int32).tofile(f)
        np.asarray(rp, np.int32).tofile(f)
        np.asarray(ci, np.int32).tofile(f)
        np.asarray(va, np.float64).tofile(f)
        np.asarray(part, np.int32).tofile(f)
    subprocess.check_call([probe, fin, fout])
    raw = np.fromfile(fout, dtype=np.uint8)
    os.remove(fin)
    os.remove(fout)
    pos = 0

    def i32():
        nonlocal pos
        v = int(raw[pos:pos + 4].view(np.int32)[0])
        pos += 4
        return v

    st = i32()
    out = {"status": st}
    while True:
        ln = i32()
        if ln == 0:
            break
        name = bytes(raw[pos:pos + ln]).decode()
        pos += ln
        if st != 0:
            out["error"] = name
            continue
        cnt = i32()
        out[name] = raw[pos:pos + 4 * cnt].view(np.int32).copy()
        pos += 4 * cnt
    return out


def _rows(A):
    n, rp, ci, _ = A
    return [ci[rp[i]:rp[i + 1]] for i in range(n)]


def _pos(A, i, j):
    n, rp, ci, _ = A
    seg = ci[rp[i]:rp[i + 1]]
    t = np.searchsorted(seg, j)
    return int(rp[i] + t) if t < len(seg) and seg[t] == j else -1


def _block_graph(A, part, iface, b, p, members, c_solver):
    """Edges (i, j), i < j, of block b's graph, original indices."""
    rows = _rows(A)
    mem = set(int(x) for x in members)
    edges = set()
    for i in mem:
        for j in rows[i]:
            j = int(j)
            if j != i and j in mem and (b < p or c_solver == 0 or (c_solver == 1 and part[i] == part[j])):
                edges.add((min(i, j), max(i, j)))
            if b < p and iface[j]:
                for r in rows[j]:
                    r = int(r)
                    if r != i and not iface[r]:
                        assert r in mem
                        edges.add((min(i, r), max(i, r)))
    return edges


def _two_colour(nodes, edges):
    """BFS 2-colouring from the lowest node of each component (None if odd cycle)."""
    adj = {v: [] for v in nodes}
    for a, b in edges:
        adj[a].append(b)
        adj[b].append(a)
    col = {}
    for s in sorted(nodes):
        if s in col:
            continue
        col[s] = 0
        queue = [s]
        while queue:
            u = queue.pop(0)
            for v in sorted(adj[u]):
                if v not in col:
                    col[v] = 1 - col[u]
                    queue.append(v)
                elif col[v] == col[u]:
                    return None
    return col


def _level_pairs(order, edges, k):
    """Entries (later, earlier) of the level-k incomplete factor for the
    elimination order `order` (a list of nodes): the graph's edges have level
    0; pivot t gives each pair of its later neighbours i, j the level
    lev(i,t) + lev(j,t) + 1, the smallest counting, kept up to k."""
    pos = {v: e for e, v in enumerate(order)}
    col = {v: {} for v in order}            # column t -> {later row: level}
    for a, b in edges:
        lo, hi = (a, b) if pos[a] < pos[b] else (b, a)
        col[lo][hi] = 0
    out = set()
    for t in order:
        ent = sorted(col[t].items(), key=lambda kv: pos[kv[0]])
        for i, lv in ent:
            out.add((i, t))
        for x in range(len(ent)):
            for y in range(x):
                (i, li), (j, lj) = ent[x], ent[y]
                cand = li + lj + 1
                if cand <= k and cand < col[j].get(i, k + 1):
                    col[j][i] = cand
    return out


def check_plan(P, A, part, p, factor, c_order, b_order, c_solver, fill_level=0):
    n, rp, ci, va = A
    rows = _rows(A)
    part = np.asarray(part)
    iface = np.array([bool(np.any(part[rows[i]] != part[i])) for i in range(n)])
    sc = P["scalars"]
    s, m = int(iface.sum()), n - int(iface.sum())
    assert (sc[0], sc[1], sc[2], sc[3]) == (n, p, s, m)
    perm, iperm, b0 = P["perm"], P["iperm"], P["blk_row0"]
    assert np.array_equal(np.sort(perm), np.arange(n)) and np.array_equal(iperm[perm], np.arange(n))
    for b in range(p + 1):
        want = np.flatnonzero(iface) if b == p else np.flatnonzero((part == b) & ~iface)
        assert np.array_equal(np.sort(perm[b0[b]:b0[b + 1]]), want)
    assert np.array_equal(perm[m:][np.argsort(P["iface_rank"])], np.flatnonzero(iface))
    # factor pattern, value sources, E Ehat^T terms
    f_rp, f_ci = P["f_rp"], P["f_ci"]
    level = np.zeros(n, np.int64)
    for b in range(p + 1):
        mem = perm[b0[b]:b0[b + 1]]
        order = b_order if b < p else c_order
        edges = _block_graph(A, part, iface, b, p, mem, c_solver)
        lower = set()
        for g in range(b0[b], b0[b + 1]):
            cols = f_ci[f_rp[g]:f_rp[g + 1]]
            assert cols[-1] == g and np.all(np.diff(cols) > 0) and np.all(cols[:-1] >= b0[b])
            for c in cols[:-1]:
                lower.add((g, int(c)))
            level[g] = 1 + max((level[c] for c in cols[:-1]), default=-1)
        pairs = {(int(iperm[max(i, j)]), int(iperm[min(i, j)])) for i, j in edges}
        pairs = {(max(a, c), min(a, c)) for a, c in pairs}
        if factor == 0 and fill_level == 0:
            assert lower == pairs
        elif factor == 0:
            # level-of-fill pattern in the block's elimination order
            nodes = [int(x) for x in mem]
            if order == 0:
                eo = sorted(nodes)
            else:
                col = _two_colour(set(nodes), edges)
                eo = None if col is None else sorted(nodes, key=lambda v: (col[v], v))
            if eo is not None:
                want = {(int(iperm[i]), int(iperm[j])) for i, j in _level_pairs(eo, edges, fill_level)}
                assert pairs <= want and lower == want
        else:
            # exact: the pattern of a dense Cholesky factor of a matrix with
            # the block's graph (random weights, diagonally dominant), in the
            # elimination order that the device order refines
            assert pairs <= lower
            nb = len(mem)
            loc = {int(g): t for t, g in enumerate(range(b0[b], b0[b + 1]))}
            rng = np.random.default_rng(0)
            M = np.eye(nb) * (4.0 * nb)
            for a, c in pairs:
                w = rng.uniform(0.5, 1.0)
                M[loc[a], loc[c]] = M[loc[c], loc[a]] = -w
            Lc = np.linalg.cholesky(M)
            dense = {(a, c) for a in range(b0[b], b0[b + 1]) for c in range(b0[b], a)
                     if abs(Lc[loc[a], loc[c]]) > 1e-300}
            assert lower == dense
        # elimination order on every edge
        if order == 0:
            assert all(perm[g] > perm[c] for g, c in pairs)
        else:
            col = _two_colour(set(int(x) for x in mem), edges)
            if col is not None:
                assert all(col[int(perm[c])] == 0 and col[int(perm[g])] == 1 for g, c in pairs)
                if b == p and edges and factor == 0 and fill_level == 0:
                    assert sc[6] == 2 and sc[5] == 2   # two colours, two levels
    f_src = P["f_src"]
    for g in range(n):
        i = int(perm[g])
        for q in range(f_rp[g], f_rp[g + 1]):
            assert f_src[q] == _pos(A, i, int(perm[f_ci[q]]))
    cd = P["f_cdiag"]
    assert np.array_equal(np.flatnonzero(cd), f_rp[m + 1:n + 1] - 1)
    f_prp, f_pa, f_pb = P["f_prp"], P["f_pa"], P["f_pb"]
    for g in range(m):
        i = int(perm[g])
        for q in range(f_rp[g], f_rp[g + 1]):
            r = int(perm[f_ci[q]])
            want = sorted((_pos(A, i, int(j)), _pos(A, r, int(j)))
                          for j in rows[i] if iface[j] and _pos(A, r, int(j)) >= 0)
            got = sorted(zip(f_pa[f_prp[q]:f_prp[q + 1]], f_pb[f_prp[q]:f_prp[q + 1]]))
            assert [tuple(map(int, t)) for t in got] == want
    # levels: records, monotone inside blocks, schedule, descriptors, chunks
    lr0, lnr, bl0 = P["lvl_row0"], P["lvl_nrows"], P["blk_lvl0"]
    for b in range(p + 1):
        assert np.all(np.diff(level[b0[b]:b0[b + 1]]) >= 0)
        for L, rec in enumerate(range(bl0[b], bl0[b + 1])):
            assert np.all(level[lr0[rec]:lr0[rec] + lnr[rec]] == L) and lnr[rec] > 0
        assert sum(lnr[bl0[b]:bl0[b + 1]]) == b0[b + 1] - b0[b]
    assert np.array_equal(P["fl_rows"], np.argsort(level, kind="stable"))
    assert np.array_equal(P["fl_ptr"], np.concatenate([[0], np.cumsum(np.bincount(level))]))
    seen = np.zeros(n, np.int64)
    ch, cap = P["chunks"].reshape(-1, 4), P["ch_all_ptr"]
    for L in range(len(cap) - 1):
        for t in range(cap[L], cap[L + 1]):
            rec, first, cnt, _ = ch[t]
            assert 0 < cnt <= 256 and first + cnt <= lnr[rec]
            rr = np.arange(lr0[rec] + first, lr0[rec] + first + cnt)
            assert np.all(level[rr] == L)
            seen[rr] += 1
    assert np.all(seen == 1)
    # sliced-ELL solve layouts and their slot maps
    slot = P["row_slot"]
    upper = [[] for _ in range(n)]
    for g in range(n):
        for q in range(f_rp[g], f_rp[g + 1] - 1):
            upper[int(f_ci[q])].append((g, q))
    map_l, map_u = P["map_l"], P["map_u"]
    for g in range(n):
        sl, ln = divmod(int(slot[g]), 32)
        low = f_ci[f_rp[g]:f_rp[g + 1] - 1]
        for kk in range(P["l_sw"][sl]):
            at = P["l_soff"][sl] + kk * 32 + ln
            if kk < len(low):
                assert P["l_col"][at] == low[kk] and map_l[f_rp[g] + kk] == at
            else:
                assert level[P["l_col"][at]] == 0
        up = upper[g]
        for kk in range(P["u_sw"][sl]):
            at = P["u_soff"][sl] + kk * 32 + ln
            if kk < len(up):
                assert P["u_col"][at] == up[kk][0] and map_u[up[kk][1]] == at
            else:
                blk = np.searchsorted(b0, P["u_col"][at], side="right") - 1
                assert level[P["u_col"][at]] == level[b0[blk]:b0[blk + 1]].max()
        assert map_l[f_rp[g + 1] - 1] == -1 and map_u[f_rp[g + 1] - 1] == -1
    if len(P["lv_desc"]):
        dsc = P["lv_desc"].reshape(-1, 4)
        assert np.array_equal(dsc[:, 0], P["fl_rows"]) and np.array_equal(P["lv_ptr"], P["fl_ptr"])
        for r, lo_, uo, w in dsc:
            sl, ln = divmod(int(slot[r]), 32)
            assert lo_ == P["l_soff"][sl] + ln and uo == P["u_soff"][sl] + ln
            assert (w & 0xFFFF) == f_rp[r + 1] - f_rp[r] - 1 and (w >> 16) == len(upper[r])
    # Ehat, Ehat^T and the SpMV layout
    ent_e, ent_et = set(), set()
    for g in range(m):
        for t in range(P["eh_rp"][g], P["eh_rp"][g + 1]):
            j = int(P["eh_ci"][t])
            q = int(P["eh_src"][t])
            assert ci[q] == perm[m + j] and rp[perm[g]] <= q < rp[perm[g] + 1]
            ent_e.add((g, j))
    for j in range(s):
        for t in range(P["eht_rp"][j], P["eht_rp"][j + 1]):
            ent_et.add((int(P["eht_ci"][t]), j))
    want_e = {(int(iperm[i]), int(iperm[j]) - m) for i in range(n) if not iface[i] for j in rows[i] if iface[j]}
    assert ent_e == want_e == ent_et
    a_soff, a_sw, a_col, a_src = P["a_soff"], P["a_sw"], P["a_col"], P["a_src"]
    for g in range(n):
        sl, ln = divmod(g, 32)
        got = {(int(a_col[a_soff[sl] + kk * 32 + ln]), int(a_src[a_soff[sl] + kk * 32 + ln]))
               for kk in range(a_sw[sl]) if a_src[a_soff[sl] + kk * 32 + ln] >= 0}
        i = int(perm[g])
        assert got == {(int(iperm[ci[q]]), q) for q in range(rp[i], rp[i + 1])}


CASES = {
    "2d_20x16_natural": lambda: (W.laplacian((20, 16)),) + W.box_partition((20, 16), (2, 2)) + (0, 0, 0, 0),
    "2d_20x16_multicolour": lambda: (W.laplacian((20, 16)),) + W.box_partition((20, 16), (2, 2)) + (0, 1, 1, 0),
    "2d_20x16_mixed_orders": lambda: (W.laplacian((20, 16)),) + W.box_partition((20, 16), (3, 2)) + (0, 1, 0, 0),
    "3d_12_multicolour": lambda: (W.laplacian((12, 12, 12)),) + W.box_partition((12, 12, 12), (2, 2, 2))
    + (0, 1, 1, 0),
    "3d_16_random_cuts": lambda: (W.laplacian((16, 16, 16)),) + W.random_cut_partition(16, 2, 0, 6, 10)
    + (0, 0, 1, 0),
    "9pt_14_ehat_fill": lambda: (W.nine_point(14, 0.0),) + W.box_partition((14, 14), (2, 2)) + (0, 1, 0, 0),
    "2d_12_exact": lambda: (W.laplacian((12, 12)),) + W.box_partition((12, 12), (2, 2)) + (1, 0, 0, 0),
    "2d_12_exact_multicolour": lambda: (W.laplacian((12, 12)),) + W.box_partition((12, 12), (2, 2)) + (1, 1, 1, 0),
    "2d_20x16_chebyshev": lambda: (W.laplacian((20, 16)),) + W.box_partition((20, 16), (2, 2)) + (0, 1, 1, 1),
    "2d_20x16_mr": lambda: (W.laplacian((20, 16)),) + W.box_partition((20, 16), (2, 2)) + (0, 1, 1, 2),
}

FILL_CASES = {
    "2d_20x16_fill1_natural": lambda: (W.laplacian((20, 16)),) + W.box_partition((20, 16), (2, 2)) + (0, 0, 0, 0, 1),
    "2d_20x16_fill2_multicolour": lambda: (W.laplacian((20, 16)),) + W.box_partition((20, 16), (2, 2))
    + (0, 1, 1, 0, 2),
    "3d_10_fill2_natural": lambda: (W.laplacian((10, 10, 10)),) + W.box_partition((10, 10, 10), (2, 2, 2))
    + (0, 0, 0, 0, 2),
    "9pt_14_fill1_natural": lambda: (W.nine_point(14, 0.0),) + W.box_partition((14, 14), (2, 2)) + (0, 0, 0, 0, 1),
    "2d_20x16_fill3_ldl": lambda: (W.shifted_laplacian((20, 16), 1.0),) + W.box_partition((20, 16), (2, 2))
    + (2, 0, 1, 0, 3),
}


@pytest.mark.parametrize("name", list(CASES))
def test_plan_matches_definitions(probe, name):
    A, part, p, factor, c_order, b_order, c_solver = CASES[name]()
    P = run_plan(probe, A, part, p, name, factor=factor, c_order=c_order, b_order=b_order, c_solver=c_solver)
    assert P["status"] == 0, P.get("error")
    check_plan(P, A, part, p, factor, c_order, b_order, c_solver)


@pytest.mark.parametrize("name", list(FILL_CASES))
def test_fill_plan_matches_definitions(probe, name):
    A, part, p, factor, c_order, b_order, c_solver, fill = FILL_CASES[name]()
    P = run_plan(probe, A, part, p, name, factor=factor, c_order=c_order, b_order=b_order, c_solver=c_solver,
                 fill_level=fill)
    assert P["status"] == 0, P.get("error")
    check_plan(P, A, part, p, 0 if factor == 2 else factor, c_order, b_order, c_solver, fill_level=fill)


def test_plan_errors(probe):
    A = W.laplacian((8, 8))
    part, p = W.box_partition((8, 8), (2, 2))
    n, rp, ci, va = A
    va2 = va.copy()
    va2[1] += 1.0
    P = run_plan(probe, (n, rp, ci, va2), part, p, "asym")
    assert P["status"] == 1 and "symmetric" in P["error"]
    P = run_plan(probe, A, np.zeros(n, np.int32), 1, "nointerface")
    assert P["status"] == 1 and "interface" in P["error"]
