"""Pins for oracle.sketch: the counter-based generator and the sketches."""

import os

import numpy as np
import pytest

from oracle import sketch

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "splitmix64.txt")


def _golden():
    rows = []
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        vals = [int(t) for t in line.split()]
        rows.append((vals[0], vals[1:]))
    return rows


def test_splitmix64_reference_outputs():
    for seed, outs in _golden():
        got = sketch.splitmix64_stream(seed, len(outs))
        assert [int(v) for v in got] == outs


def test_counter_draw_equals_stream_position():
    # draw(seed, t-1) is output t of the sequential stream
    seq = sketch.splitmix64_stream(1234567, 50)
    ctr = sketch.draw(1234567, np.arange(50, dtype=np.uint64))
    assert np.array_equal(seq, ctr)


def test_mix64_is_bijective_on_sample():
    # invert the three xorshift-multiply steps; a wrong shift breaks this
    def inv_xorshift(z, k):
        out = z.copy()
        for _ in range(64 // k + 1):
            out = z ^ (out >> np.uint64(k))
        return out

    z = np.random.default_rng(1).integers(0, 2**63, size=1000, dtype=np.uint64) * np.uint64(2) + np.uint64(1)
    y = sketch.mix64(z)
    c2 = pow(0x94D049BB133111EB, -1, 2**64)
    c1 = pow(0xBF58476D1CE4E5B9, -1, 2**64)
    with np.errstate(over="ignore"):
        t = inv_xorshift(y, 31) * np.uint64(c2)
        t = inv_xorshift(t, 27) * np.uint64(c1)
        t = inv_xorshift(t, 30)
    assert np.array_equal(t, z)


@pytest.mark.parametrize("w,s", [(64, 1), (64, 2), (96, 3), (128, 4)])
def test_countsketch_structure(w, s):
    n = 500
    W = sketch.countsketch_matrix(7, 3, 0, n, w, s).toarray()
    wb = w // s
    for b in range(s):
        blk = W[:, b * wb:(b + 1) * wb]
        # exactly one nonzero per row per block, value +-1/sqrt(s)
        assert np.array_equal((blk != 0).sum(axis=1), np.ones(n))
        assert np.allclose(np.abs(blk[blk != 0]), 1.0 / np.sqrt(s))
    # squared row norms are exactly 1 (E[W W^T] = I on the diagonal)
    assert np.allclose((W * W).sum(axis=1), 1.0)


def test_countsketch_buckets_uniform_and_signs_balanced():
    n, w, s = 200_000, 64, 2
    cols, signs = sketch.countsketch_hash(11, 0, 0, n, w, s)
    for b in range(s):
        counts = np.bincount(cols[b] - b * (w // s), minlength=w // s)
        expected = n / (w // s)
        chi2 = ((counts - expected) ** 2 / expected).sum()
        # 31 degrees of freedom: P(chi2 > 70) < 1e-4
        assert chi2 < 70.0
        assert abs(signs[b].mean()) < 5.0 / np.sqrt(n)


def test_countsketch_redraw_changes_hash():
    a = sketch.countsketch_hash(5, 2, 0, 1000, 64, 2)[0]
    b = sketch.countsketch_hash(5, 2, 1, 1000, 64, 2)[0]
    c = sketch.countsketch_hash(5, 3, 0, 1000, 64, 2)[0]
    assert (a != b).mean() > 0.8 and (a != c).mean() > 0.8


def test_countsketch_blocks_hash_independently():
    # the s blocks of one draw are independent hashes (each row has one
    # nonzero per block, at a bucket and sign of its own): two blocks put a
    # row in the same in-block bucket with probability 1/(w/s) and give it
    # the same sign half of the time
    n, w, s = 20000, 128, 2
    cols, signs = sketch.countsketch_hash(5, 2, 0, n, w, s)
    h0, h1 = cols[0], cols[1] - w // s
    assert abs((h0 == h1).mean() - 1.0 / (w // s)) < 0.01
    assert abs((signs[0] == signs[1]).mean() - 0.5) < 0.03


def test_sparse_embedding_approximates_gram():
    # eq. pdprec with Z = V^T (orthonormal rows): ||Z W W^T Z^T - I|| small for large w
    rng = np.random.default_rng(0)
    m, n = 4, 4000
    V, _ = np.linalg.qr(rng.standard_normal((n, m)))
    W = sketch.countsketch_matrix(3, 0, 0, n, 4096, 4)
    ZW = (W.T @ V).T
    err = np.linalg.norm(ZW @ ZW.T - np.eye(m), 2)
    assert err < 0.25


def test_gaussian_sketch_moments():
    n, w = 400, 256
    G = sketch.gaussian_matrix(9, 1, 0, n, w) * np.sqrt(w)
    assert abs(G.mean()) < 0.02
    assert abs(G.var() - 1.0) < 0.03
    # fourth moment of N(0,1) is 3
    assert abs((G ** 4).mean() - 3.0) < 0.15
    G2 = sketch.gaussian_matrix(9, 2, 0, n, w)
    assert not np.allclose(G / np.sqrt(w), G2)


def test_gaussian_sketch_uses_both_box_muller_outputs():
    # entries 2p and 2p+1 (flat, row-major) are the cosine and sine normals of
    # draw p: r cos(t) and r sin(t) with the same r and t, so their squares
    # add up to r^2 = -2 ln u1, and across draws the two halves are
    # uncorrelated N(0, 1) samples with the same moments
    n, w = 300, 200
    G = sketch.gaussian_matrix(5, 3, 1, n, w).reshape(-1) * np.sqrt(w)
    u1, u2 = sketch.gaussian_uniforms(5, 3, 1, n, w)
    even, odd = G[0::2], G[1::2]
    assert np.allclose(even ** 2 + odd ** 2, -2.0 * np.log(u1), rtol=1e-12)
    assert np.allclose(np.arctan2(odd, even) % (2 * np.pi), (2 * np.pi * u2) % (2 * np.pi), atol=1e-9)
    assert abs(np.corrcoef(even, odd)[0, 1]) < 0.02
    assert abs(even.var() - 1.0) < 0.03 and abs(odd.var() - 1.0) < 0.03
    # an odd width pairs entries across rows: the flat index decides
    G3 = sketch.gaussian_matrix(5, 3, 1, 7, 3).reshape(-1) * np.sqrt(3)
    v1, _ = sketch.gaussian_uniforms(5, 3, 1, 7, 3)
    assert v1.size == 11
    assert np.allclose(G3[0:20:2] ** 2 + G3[1:21:2] ** 2, -2.0 * np.log(v1[:10]), rtol=1e-12)


def test_gaussian_uniforms_are_exact_fp32_and_in_range():
    u1, u2 = sketch.gaussian_uniforms(3, 1, 0, 50, 40)
    assert np.array_equal(u1.astype(np.float32).astype(np.float64), u1)
    assert np.array_equal(u2.astype(np.float32).astype(np.float64), u2)
    assert (u1 > 0).all() and (u1 <= 1).all() and (u2 >= 0).all() and (u2 < 1).all()


def test_gaussian_sketch_subspace_embedding():
    # Section 6: a Gaussian W with w >> m is a subspace embedding (eq. pdprec)
    rng = np.random.default_rng(4)
    m, n, w = 4, 3000, 2000
    V, _ = np.linalg.qr(rng.standard_normal((n, m)))
    W = sketch.gaussian_matrix(8, 0, 0, n, w)
    G = (V.T @ W) @ (W.T @ V)
    assert np.linalg.norm(G - np.eye(m), 2) < 0.25


def _basis_rows(cols, signs, basis, w, s):
    """W_B: the rows of the CountSketch for the columns in `basis` (m x w)."""
    wb = np.zeros((len(basis), w))
    for b in range(s):
        wb[np.arange(len(basis)), cols[b, basis]] += signs[b, basis] / np.sqrt(s)
    return wb


def test_countsketch_rank_on_a_coordinate_subspace_depends_on_s():
    """Near an IPM optimum range((AD)^T) is close to the span of the m basic
    coordinates, so W embeds it only if W_B (its rows for those columns) has
    rank m.  With s = 1 two basic columns sharing a bucket already make W_B
    singular (about m^2/(2w) shared pairs at w = 4m); with s = 2 a pair sharing
    both buckets with equal sign products (or a longer cycle of shared buckets)
    does, in a few per cent of draws; with s = 4 it takes far rarer
    coincidences.  This is the failure the GPU path detects and redraws."""
    m, n, w = 128, 16384, 512
    basis = np.sort(np.random.default_rng(5).choice(n, m, replace=False))
    draws = [(k, r) for k in range(10) for r in range(4)]
    singular = {1: 0, 2: 0, 4: 0}
    for s in (1, 2, 4):
        for k, r in draws:
            cols, signs = sketch.countsketch_hash(0, k, r, n, w, s)
            sv = np.linalg.svd(_basis_rows(cols, signs, basis, w, s), compute_uv=False)
            is_singular = sv[-1] < 1e-10 * sv[0]
            singular[s] += int(is_singular)
            if s == 2:
                seen = {}
                dependent_pair = False
                for j in basis:
                    key = (int(cols[0, j]), int(cols[1, j]))
                    if key in seen:
                        i = seen[key]
                        dependent_pair |= signs[0, i] * signs[1, i] == signs[0, j] * signs[1, j]
                    seen[key] = j
                assert not dependent_pair or is_singular
    assert singular[1] == len(draws)
    assert 1 <= singular[2] <= 0.4 * len(draws), singular
    assert singular[4] == 0, singular


def test_gaussian_uniforms_reach_both_ends_of_their_grids():
    # u1 lives on {1, ..., 2^23} / 2^23 (never 0: it goes through a log) and
    # u2 on {0, ..., 2^23 - 1} / 2^23.  Over 2^24 draws every end value turns
    # up with probability 1 - e^-2 each; seed 0 shows all four, so a map that
    # is off by one grid step at either end fails here.
    u1, u2 = sketch.gaussian_uniforms(0, 0, 0, 4096, 8192)
    assert u1.size == 2 ** 24
    step = 2.0 ** -23
    assert u1.min() == step and u1.max() == 1.0
    assert u2.min() == 0.0 and u2.max() == 1.0 - step
    assert np.isfinite(np.log(u1)).all()


def test_preconditioned_condition_number_by_sketch_and_regime():
    # kappa(Q^{-1} M) of Q^{-1/2} A D at w = 4m: with spread D every sketch
    # sits near the Marchenko-Pastur value ((1 + 1/2)/(1 - 1/2))^2 = 9; near
    # the optimum (m dominant columns of D) one nonzero per row collapses
    # (two basic columns in one bucket make W_B singular) while s = 4 stays
    # within twice the Gaussian sketch
    from oracle import pcg
    m, n, w = 64, 8192, 256
    rng = np.random.default_rng(100)
    A = rng.standard_normal((m, n))

    def kappa2(AD, W):
        ADW = np.asarray((W.T @ AD.T).T) if hasattr(W, "tocsc") else AD @ W
        sv = np.linalg.svd(pcg.preconditioner(ADW).Q_mhalf @ AD, compute_uv=False)
        return (sv[0] / sv[-1]) ** 2

    spread = A * np.exp(rng.uniform(-3, 3, n))
    d = np.exp(rng.uniform(-8, -4, n))
    d[rng.choice(n, m, replace=False)] = np.exp(rng.uniform(3, 6, m))
    near = A * d
    sketches = {s: sketch.countsketch_matrix(0, 0, 0, n, w, s) for s in (1, 2, 4)}
    gauss = sketch.gaussian_matrix(0, 0, 0, n, w)
    for W in list(sketches.values()) + [gauss]:
        assert 5.0 < kappa2(spread, W) < 12.0
    k_gauss = kappa2(near, gauss)
    assert kappa2(near, sketches[1]) > 1e4
    assert kappa2(near, sketches[4]) < 2.0 * k_gauss
    assert kappa2(near, sketches[2]) > kappa2(near, sketches[4])
