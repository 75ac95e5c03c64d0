"""Race freedom and coverage of the kernels that accumulate without atomics,
checked by enumeration on the CPU (the index arithmetic restated from the
kernels; no GPU).

* The complex128 scatters (csrc/resample2d_f64.cu, csrc/resample3d_f64.cu):
  a thread owns the region points whose coordinates fall in one residue class
  (2D: column mod 16 and row mod 8 over 128 threads; 3D: (mod 4, mod 4,
  mod 8)).  For every node offset in the tile and every supported K, each
  footprint point must be written by exactly one thread, always the one that
  owns it, and inside the region.
* The register-resident gather (csrc/resample3d.cu, gather3d_reg_kernel):
  warp w holds region rows 4w .. 4w + 3 and visits the nodes whose a1 lies in
  [lo_w, hi_w]; the final sum adds the slots of exactly the warps whose rows
  meet the node's footprint.
"""
import itertools

import pytest


def _thread_2d(tid, a0, a1, K):
    """Points (row, col) that thread tid of the 2D FP64 scatter writes for a
    node at offset (a0, a1): warp w = tid >> 5, lane = tid & 31,
    c16 = lane & 15, h = lane >> 4, row residue 2w + h mod 8."""
    warp, lane = tid >> 5, tid & 31
    c16, h = lane & 15, lane >> 4
    rres = 2 * warp + h
    j1 = (c16 - a1) & 15
    if j1 >= K:
        return []
    i0s = (rres - a0) & 7
    out = []
    for k in range((K + 7) // 8):
        i0 = i0s + 8 * k
        if i0 < K:
            out.append((a0 + i0, a1 + j1))
    return out


@pytest.mark.parametrize("K", [2, 4, 6, 8, 10, 12, 14, 16])
def test_2d_f64_scatter_ownership(K):
    T = (5, 17)
    L = (T[0] + K - 1, T[1] + K - 1)
    owner = {}
    for a0, a1 in itertools.product(range(T[0]), range(T[1])):
        written = {}
        for tid in range(128):
            for pt in _thread_2d(tid, a0, a1, K):
                assert pt not in written, "two threads write one point"
                written[pt] = tid
                assert 0 <= pt[0] < L[0] and 0 <= pt[1] < L[1]
                # the owner of a point never changes from node to node
                assert owner.setdefault(pt, tid) == tid
        footprint = {(a0 + i, a1 + j) for i in range(K) for j in range(K)}
        assert set(written) == footprint


def _thread_3d(tid, a, K):
    r0, r1, c2 = tid >> 5, (tid >> 3) & 3, tid & 7
    j2 = (c2 - a[2]) & 7
    if j2 >= K:
        return []
    i0s, i1s = (r0 - a[0]) & 3, (r1 - a[1]) & 3
    out = []
    for k0 in range((K + 3) // 4):
        for k1 in range((K + 3) // 4):
            i0, i1 = i0s + 4 * k0, i1s + 4 * k1
            if i0 < K and i1 < K:
                out.append((a[0] + i0, a[1] + i1, a[2] + j2))
    return out


@pytest.mark.parametrize("K", [2, 4, 6, 8])
def test_3d_f64_scatter_ownership(K):
    T = (3, 4, 9)
    owner = {}
    for a in itertools.product(range(T[0]), range(T[1]), range(T[2])):
        written = {}
        for tid in range(128):
            pts = _thread_3d(tid, a, K)
            assert len(pts) <= 4
            for pt in pts:
                assert pt not in written, "two threads write one point"
                written[pt] = tid
                assert all(0 <= pt[d] < T[d] + K - 1 for d in range(3))
                assert owner.setdefault(pt, tid) == tid
        footprint = {(a[0] + i, a[1] + j, a[2] + k) for i in range(K) for j in range(K) for k in range(K)}
        assert set(written) == footprint


@pytest.mark.parametrize("K,T1", [(8, 9), (12, 5)])
def test_register_gather_warp_visits(K, T1):
    for a1 in range(T1):
        rows = set(range(a1, a1 + K))
        assert max(rows) < 16
        for w in range(4):
            lo, hi = max(0, 4 * w - (K - 1)), min(8, 4 * w + 3)
            visits = lo <= a1 <= hi                              # the node loop's a1 run
            summed = a1 >= max(0, 4 * w - (K - 1)) and a1 <= 4 * w + 3   # the final pass
            meets = bool(rows & set(range(4 * w, 4 * w + 4)))
            assert visits == meets == summed
