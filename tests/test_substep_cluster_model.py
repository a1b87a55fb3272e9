"""A model of k_substep_cluster<C> (csrc/step.cu): how the 64-body blocks of the multi-kernel
substep (k_kick, k_rebuild, k_shift, k_drift) are dealt out over a cluster of C CTAs of G groups,
the index ranges every phase touches, and the sums it forms. CPU only.

The kernel's rules, restated:
- nblk = ceil(npad / 64) blocks; a pass of the cluster covers C G blocks, and there are
  ceil(nblk / (C G)) passes; group g of CTA r takes block (it C + r) G + g in pass it;
- a group is 3 x 64 threads, thread (c, b): component c of body 64 blk + b (index order in the
  kick, shift and drift; bylev[64 blk + b] in the walks);
- the element-wise phases touch w < npad (kick and drift) or w < n (shift); the walks take
  i < n;
- a block's partial is the sum of its 64 bodies' terms by a shuffle tree in each of two warps,
  then the two warp sums added; the cluster adds the nblk partials in sum_partials' order
  (lane l sums blocks l, l + 32, ..., then a shuffle tree over the lanes).
"""
import numpy as np
import pytest

BLOCK = 64


def assignment(npad, C, G):
    nblk = -(-npad // BLOCK)
    passes = -(-nblk // (C * G))
    owner = {}
    for it in range(passes):
        for r in range(C):
            for g in range(G):
                blk = (it * C + r) * G + g
                if blk < nblk:
                    assert blk not in owner
                    owner[blk] = (r, g, it)
    return nblk, owner


@pytest.mark.parametrize("n,T", [(257, 32), (600, 32), (1000, 64), (2050, 32), (2050, 128), (4000, 64),
                                 (4096, 128)])
@pytest.mark.parametrize("C", [2, 4, 8])
def test_every_block_and_body_has_one_owner(n, T, C):
    npad = -(-n // T) * T
    G = min(5, -(-(-(-npad // BLOCK)) // C))
    nblk, owner = assignment(npad, C, G)
    assert sorted(owner) == list(range(nblk))
    # element-wise phases: every w < npad is touched once, by one (CTA, group, pass), per component
    seen = np.zeros(npad, int)
    for blk in owner:
        for b in range(BLOCK):
            w = blk * BLOCK + b
            if w < npad:
                seen[w] += 1
    assert (seen == 1).all()
    # shared-memory indices: 3 npad planes, 3 nblk and nblk partials, 5 groups of scratch
    assert max(blk * 3 + 2 for blk in owner) < 3 * nblk
    assert G <= 5 and 6 * (G - 1) + 5 < 30


def warp_tree(x):
    """The shuffle-down tree over 32 lanes: lane 0's result."""
    x = list(x)
    o = 16
    while o:
        x = [x[l] + (x[l + o] if l + o < 32 else 0.0) for l in range(32)]
        o //= 2
    return x[0]


def block_sum64(vals):
    """block_sum of k_shift / k_rebuild over 64 threads: warp trees, then warp 0 reduces the two
    warp sums (padded with zeros) by the same tree."""
    s0, s1 = warp_tree(vals[:32]), warp_tree(vals[32:])
    return warp_tree([s0, s1] + [0.0] * 30)


def test_two_warp_sums_equal_block_sum():
    """The kernel adds the two warp sums directly; block_sum's second tree adds zeros to them first,
    which changes nothing, so the block partials are bit-identical."""
    rng = np.random.default_rng(5)
    for _ in range(2000):
        v = rng.standard_normal(64) * 10.0 ** rng.integers(-20, 20, 64)
        s0, s1 = warp_tree(v[:32]), warp_tree(v[32:])
        assert s0 + s1 == block_sum64(v)


def test_sum_partials_order():
    """The cluster's sum of nblk partials is sum_partials' order: identical for every CTA."""
    rng = np.random.default_rng(6)
    for nblk in (5, 33, 64, 65, 130):
        p = rng.standard_normal(nblk)
        lanes = []
        for l in range(32):
            s = 0.0
            for bb in range(l, nblk, 32):
                s += p[bb]
            lanes.append(s)
        a = warp_tree(lanes)
        b = warp_tree(lanes)
        assert a == b and np.isclose(a, p.sum(), rtol=1e-13, atol=1e-13)
