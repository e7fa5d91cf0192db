"""Pins of the PMM oracle (Sec. 3.4, Eq. 11) against closed forms, invariants
and brute force; no GPU."""
import math

import numpy as np
import pytest

from oracle import pmm

R = pmm.RATIO


def _blocks_to_map(cells, Hc, Wc, ratio=R, jitter=None):
    """Fine map (C, Hc*ratio, Wc*ratio) whose block (cy, cx) holds the vector cells[cy*Wc+cx] everywhere
    (plus optional per-pixel jitter)."""
    C = cells.shape[1]
    F = np.repeat(np.repeat(cells.T.reshape(C, Hc, Wc), ratio, axis=1), ratio, axis=2).astype(np.float32)
    if jitter is not None:
        F = (F + jitter).astype(np.float32)
    return F


def test_coarse_unit_means_match_plain_loops():
    # the definition's coarse vectors: block means and norms by plain Python float loops
    g = np.random.default_rng(10)
    F = g.standard_normal((5, 16, 24)).astype(np.float32)
    F[:, 8:16, 0:8] = 0.0  # one zero cell stays zero
    u = pmm.coarse_unit_means(F)
    C, H, W = F.shape
    for cy in range(H // R):
        for cx in range(W // R):
            m = []
            for c in range(C):
                s = 0.0
                for dy in range(R):
                    for dx in range(R):
                        s += float(F[c, cy * R + dy, cx * R + dx])
                m.append(s / 64.0)
            nrm = math.sqrt(sum(v * v for v in m))
            exp = [v / nrm if nrm > 0 else 0.0 for v in m]
            np.testing.assert_allclose(u[cy * (W // R) + cx], exp, rtol=1e-13, atol=1e-15)
    assert not u[1 * (W // R) + 0].any()
    nz = np.linalg.norm(u, axis=1)
    np.testing.assert_allclose(nz[nz > 0], 1.0, rtol=1e-14)
    # scaling a map leaves its unit means unchanged
    np.testing.assert_allclose(pmm.coarse_unit_means((F * np.float32(4.0)).astype(np.float32)), u, rtol=1e-14,
                               atol=1e-15)


def test_bf16_precision_layer_matches_binary32_brute_force():
    # plain loops over np.float32 scalars in the stated order give the same bits
    g = np.random.default_rng(0)
    F = g.standard_normal((4, 16, 24)).astype(np.float32)
    codes = pmm.coarse_codes_bf16(F)
    C, H, W = F.shape
    for cy in range(H // R):
        for cx in range(W // R):
            m = []
            for c in range(C):
                s = np.float32(0.0)
                for dy in range(R):
                    for dx in range(R):
                        s = np.float32(s + F[c, cy * R + dy, cx * R + dx])
                m.append(np.float32(s * np.float32(1.0 / 64)))
            ss = np.float32(0.0)
            for v in m:
                ss = np.float32(ss + np.float32(v * v))
            n = np.float32(math.sqrt(float(ss)))  # sqrt of a float32 value, correctly rounded to float32
            u = np.array([np.float32(v / n) for v in m], np.float32)
            np.testing.assert_array_equal(codes[cy * (W // R) + cx], pmm._bf16_round_bits(u))


def test_bf16_precision_layer_rounds_the_unit_means():
    g = np.random.default_rng(1)
    F = g.standard_normal((32, 40, 64)).astype(np.float32)
    codes = pmm.bf16_to_f64(pmm.coarse_codes_bf16(F))
    np.testing.assert_allclose(codes, pmm.coarse_unit_means(F), rtol=2 ** -8, atol=1e-6)  # 8 significant bits
    # zero map: zero codes; constant map: one code everywhere
    assert not pmm.coarse_codes_bf16(np.zeros((32, 16, 16), np.float32)).any()
    const = np.broadcast_to(g.standard_normal((32, 1, 1)).astype(np.float32), (32, 16, 16))
    cc = pmm.coarse_codes_bf16(const)
    assert (cc == cc[0]).all()


def test_decision_changes_counts_a_flip_of_the_bf16_layer():
    # query cell 0 and rendered cells 0 and 1 are unit vectors in one plane, at
    # angles whose cosines with the query differ by 3.4e-4 (rendered cell 0
    # nearer); rounded to bf16 (8 significant bits) cell 1 comes out 2e-3 nearer
    C = 32
    a, t0, t1 = 0.5915012152990735, 1.0673854012188002, 1.0699896623145377
    q = np.zeros(C)
    q[0], q[1] = a, math.sqrt(1 - a * a)
    r0 = np.zeros(C)
    r0[0], r0[1] = math.cos(t0), math.sin(t0)
    r1 = np.zeros(C)
    r1[0], r1[1] = math.cos(t1), math.sin(t1)
    fill = np.eye(C)[3:5]  # two more cells on each side, matching each other
    Fq = _blocks_to_map(np.stack([q, fill[0], fill[1]]), 1, 3)
    Fr = _blocks_to_map(np.stack([r0, r1, fill[0], fill[1]]), 1, 4)
    d = pmm.coarse_pmm(Fq, Fr)
    b = pmm.coarse_pmm_bf16(Fq, Fr)
    assert d["row_best"][0] == 0 and b["row_best"][0] == 1
    ch = pmm.decision_changes(b, d)
    assert ch["row"] == pytest.approx(1 / 3)
    same = pmm.decision_changes(d, d)
    assert same["row"] == same["col"] == same["matches"] == 0.0


def test_dual_softmax_is_product_of_row_and_column_softmax():
    g = np.random.default_rng(2)
    M = g.uniform(-1, 1, (5, 7))
    logP, r, c = pmm.log_dual_softmax(M, 0.1)
    for i in range(5):
        for j in range(7):
            row = math.exp(M[i, j] / 0.1) / sum(math.exp(M[i, k] / 0.1) for k in range(7))
            col = math.exp(M[i, j] / 0.1) / sum(math.exp(M[k, j] / 0.1) for k in range(5))
            assert logP[i, j] == pytest.approx(math.log(row * col), rel=1e-12)
    np.testing.assert_allclose(np.exp(M / 0.1 - r[:, None]).sum(axis=1), 1.0, rtol=1e-12)
    np.testing.assert_allclose(np.exp(M / 0.1 - c[None, :]).sum(axis=0), 1.0, rtol=1e-12)


def test_orthonormal_codes_closed_form():
    # cells carry distinct unit basis vectors (exact in bf16): M = I, so every cell matches
    # itself with P = e^{2/tau} / (e^{1/tau} + N - 1)^2 and off-diagonal 1 / (e^{1/tau} + N - 1)^2
    Hc, Wc, C = 3, 4, 32
    N = Hc * Wc
    cells = np.eye(C)[:N] * 0.7
    F = _blocks_to_map(cells, Hc, Wc)
    out = pmm.coarse_pmm(F, F)
    np.testing.assert_array_equal(out["M"], np.eye(N))
    np.testing.assert_array_equal(pmm.coarse_pmm_bf16(F, F)["M"], np.eye(N))
    np.testing.assert_array_equal(out["matches"], np.stack([np.arange(N)] * 2, 1))
    z = math.exp(1 / pmm.TAU) + N - 1
    np.testing.assert_allclose(out["prob"], math.exp(2 / pmm.TAU) / z ** 2, rtol=1e-12)
    logP, _, _ = pmm.log_dual_softmax(out["M"])
    np.testing.assert_allclose(np.exp(logP[0, 1]), 1 / z ** 2, rtol=1e-12)


def test_mnn_brute_force():
    g = np.random.default_rng(3)
    for _ in range(20):
        L = g.standard_normal((6, 9))
        m = pmm.mnn(L)
        exp = []
        for i in range(6):
            j = max(range(9), key=lambda k: (L[i, k], -k))
            ib = max(range(6), key=lambda k: (L[k, j], -k))
            if ib == i:
                exp.append((i, j))
        np.testing.assert_array_equal(m["matches"], np.asarray(exp, np.int64).reshape(-1, 2))


def test_permuting_rendered_cells_permutes_matches():
    g = np.random.default_rng(4)
    Hc, Wc, C = 4, 5, 32
    cells = g.standard_normal((Hc * Wc, C))
    Fq = _blocks_to_map(cells, Hc, Wc, jitter=0.05 * g.standard_normal((C, Hc * R, Wc * R)))
    perm = g.permutation(Hc * Wc)
    Fr = _blocks_to_map(cells[perm], Hc, Wc, jitter=0.05 * g.standard_normal((C, Hc * R, Wc * R)))
    out = pmm.coarse_pmm(Fq, Fr)
    # rendered cell k holds query cell perm[k]: every query cell i matches inv[i]
    inv = np.argsort(perm)
    assert len(out["matches"]) == Hc * Wc
    np.testing.assert_array_equal(out["matches"][:, 1], inv[out["matches"][:, 0]])


def test_fine_windows_match_themselves():
    g = np.random.default_rng(5)
    C, Hc, Wc = 32, 2, 3
    F = g.standard_normal((C, Hc * R, Wc * R)).astype(np.float32)
    coarse = np.stack([np.arange(Hc * Wc)] * 2, 1)
    fine = pmm.fine_pmm(F, F, coarse)
    assert len(fine["matches"]) == Hc * Wc * R * R
    np.testing.assert_array_equal(fine["matches"][:, 1], fine["matches"][:, 2])
    assert not fine["flag"].any()
    # a shifted rendered window still pairs pixels by content
    Fr = np.roll(F, 1, axis=2)  # rendered pixel x holds query pixel x - 1
    fine2 = pmm.fine_pmm(F, Fr, np.array([[0, 0]]))
    W = Wc * R
    q, r = fine2["matches"][:, 1], fine2["matches"][:, 2]
    inner = (q % W) < R - 1  # query pixels whose shifted copy stays inside the window
    np.testing.assert_array_equal(r[inner], q[inner] + 1)


def test_chunked_equals_dense():
    # the blocked form used at full image size gives the dense form's results
    g = np.random.default_rng(7)
    cells = g.standard_normal((9 * 11, 32))
    Fq = _blocks_to_map(cells, 9, 11, jitter=0.3 * g.standard_normal((32, 72, 88)))
    Fr = _blocks_to_map(cells[g.permutation(99)], 9, 11, jitter=0.3 * g.standard_normal((32, 72, 88)))
    for d, c in ((pmm.coarse_pmm(Fq, Fr), pmm.coarse_pmm_chunked(Fq, Fr, chunk=16)),
                 (pmm.coarse_pmm_bf16(Fq, Fr), pmm.coarse_pmm_chunked(Fq, Fr, chunk=16, bf16=True))):
        for k in ("row_best", "col_best", "matches"):
            np.testing.assert_array_equal(c[k], d[k])
        for k in ("lse_row", "lse_col", "row_gap", "col_gap", "prob"):
            np.testing.assert_allclose(c[k], d[k], rtol=1e-12, atol=1e-12)
