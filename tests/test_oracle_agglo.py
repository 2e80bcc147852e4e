"""Pins of the oracle's mesh coarsening (Sec. 4.1 of the paper, Algorithm 1): the hash formula,
first-wins selection, greedy pairwise matching, and the partition / geometry invariants."""
import numpy as np
import pytest

import meshgen as mg


def test_hash_formula_values(orc):
    """Eq. hash value h = [23 (N_l + N_r) + N_l N_r] mod N_f.  The paper's worked example
    (10, 12, N_f = 100) prints 5, which the printed formula does not give: 23*22 + 120 = 626 and
    626 mod 100 = 26.  The formula is taken as authoritative."""
    assert orc.face_hash(10, 12, 100) == 26
    assert orc.face_hash(10, 12, 100) != 5
    assert orc.face_hash(0, 1, 7) == 23 % 7
    assert orc.face_hash(3_000_000, 4_000_000, 9_999_991) == (23 * 7_000_000 + 12_000_000_000_000) % 9_999_991


def test_splitmix64_reference_values(orc):
    """splitmix64 output for seeds 0 and 1 (the published generator's first outputs)."""
    assert orc.splitmix64(0) == 0xE220A8397B1DCDAF
    assert orc.splitmix64(0x9E3779B97F4A7C15) == 0x6E789E6AA1B965F4


def _levels(orc, mesh, **kw):
    M = orc.Mesh(mesh)
    S = orc.Solver(M, orc.params(**kw))
    return M, S


@pytest.mark.parametrize("mk", [lambda: mg.periodic_box(8), lambda: mg.wall_box(12, 8, 10, n_prism=4),
                                lambda: mg.scale_box(8)])
def test_partition_and_volume_invariants(orc, mk):
    mesh = mk()
    M, S = _levels(orc, mesh, n_levels=3)
    prev = dict(S.level(0))
    # level 1 aggregates the coarsening's own geometry of the fine level
    prev["vol"], prev["ctr"], _, _ = M.coarsening_geometry()
    for lev in (1, 2):
        L = S.level(lev)
        m = L["map"]
        assert m.shape == (prev["nc"],)
        assert m.min() == 0 and m.max() == L["nc"] - 1
        assert len(np.unique(m)) == L["nc"]  # every coarse cell non-empty, ids contiguous
        counts = np.bincount(m, minlength=L["nc"])
        assert counts.max() <= 4  # two pairwise passes per level
        assert L["nc"] < prev["nc"]
        vsum = np.bincount(m, weights=prev["vol"], minlength=L["nc"])
        np.testing.assert_allclose(L["vol"], vsum, rtol=1e-14)
        csum = np.stack([np.bincount(m, weights=prev["vol"] * prev["ctr"][:, d], minlength=L["nc"]) for d in range(3)], 1)
        np.testing.assert_allclose(L["ctr"], csum / vsum[:, None], rtol=0, atol=1e-14)
        # coarse faces: interior faces oriented L < R, closure of every coarse cell
        fL, fR, tag, Sn = L["fL"], L["fR"], L["tag"], L["Sn"]
        inter = (fR >= 0) & (tag == -1)
        assert np.all(fL[inter] < fR[inter])
        clos = np.zeros((L["nc"], 3))
        np.add.at(clos, fL, Sn)
        np.add.at(clos, fR[fR >= 0], -Sn[fR >= 0])
        assert np.abs(clos).max() < 1e-14
        # members of a coarse cell are connected through interior faces of the finer level
        pf = (prev["fR"] >= 0) & (prev["tag"] == -1)
        same = m[prev["fL"][pf]] == m[prev["fR"][pf]]
        linked = np.bincount(m[prev["fL"][pf][same]], minlength=L["nc"])
        assert np.all(linked[counts > 1] >= counts[counts > 1] - 1)
        prev = L


def test_single_pass_is_first_wins_selection_and_greedy_matching(orc):
    """With one pass and no skewness limit, the merged pairs are exactly the greedy matching (in
    ascending face order) of the faces whose hash value appears for the first time."""
    mesh = mg.periodic_box(6)
    M, S = _levels(orc, mesh, n_levels=2, passes_per_level=1, skew_min=0.0)
    L0, L1 = S.level(0), S.level(1)
    cand = np.nonzero((L0["fR"] >= 0) & (L0["tag"] == -1))[0]
    nf = len(cand)
    a, b = L0["fL"][cand].astype(np.uint64), L0["fR"][cand].astype(np.uint64)
    h = (np.uint64(23) * (a + b) + a * b) % np.uint64(nf)
    _, first = np.unique(h, return_index=True)
    selected = np.sort(cand[first])
    # brute-force greedy matching over the selected faces
    partner = -np.ones(L0["nc"], int)
    for f in selected:
        l, r = L0["fL"][f], L0["fR"][f]
        if partner[l] < 0 and partner[r] < 0:
            partner[l], partner[r] = r, l
    m = L1["map"]
    for c in range(L0["nc"]):
        if partner[c] >= 0:
            assert m[c] == m[partner[c]]
    assert L1["nc"] == L0["nc"] - int((partner >= 0).sum()) // 2
    # numbering by the smallest member
    reps = [c for c in range(L0["nc"]) if partner[c] < 0 or c < partner[c]]
    assert np.array_equal(m[reps], np.arange(L1["nc"]))


def test_impossible_skew_limit_merges_nothing(orc):
    mesh = mg.periodic_box(5)
    M, S = _levels(orc, mesh, n_levels=2, skew_min=1.01)
    L1 = S.level(1)
    assert L1["nc"] == M.nc
    assert np.array_equal(L1["map"], np.arange(M.nc))


def test_seeded_relabelling_gives_another_valid_partition(orc):
    mesh = mg.periodic_box(6)
    _, S0 = _levels(orc, mesh, n_levels=2)
    _, S1 = _levels(orc, mesh, n_levels=2, agglo_seed=1)
    m0, m1 = S0.level(1)["map"], S1.level(1)["map"]
    assert not np.array_equal(m0, m1)
    assert len(np.unique(m1)) == m1.max() + 1
