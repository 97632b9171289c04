"""Host check of the one-launch-per-pass batch's work tables and CTA placement
(col_batched.cu, k_row_batched, the tables of csar_batch_create), for every size the
batched kernels serve, before any of it runs on a GPU: every column tile of every patch is
transformed by exactly one group of P_e CTAs inside one 4-CTA cluster (peers and exchange
ranks inside the cluster, no CTA without a tile, so every cluster-wide barrier has all its
CTAs), the per-CTA partial-sum slots are those of the per-patch launch, and every row of
every patch belongs to exactly one range CTA of 8192 values.  Mirrors the formulas; no
GPU needed."""
import itertools

import pytest

SIZES = (512, 1024, 2048, 4096)
CLUSTER = 4
E = 4096           # values per column CTA in a batch


def batch_col_p(na):
    return {512: 1, 1024: 1, 2048: 2, 4096: 4}.get(na, 0)


def col_w(n, p, e):
    return max(1, min(16, e * p // n))


def row_w(n):
    return 1 if n >= 8192 else 8192 // n


@pytest.mark.parametrize("na,nr", list(itertools.product(SIZES, SIZES)))
def test_column_tile_groups(na, nr):
    p = batch_col_p(na)
    w = col_w(na, p, E)
    assert w * 8 % 32 == 0 and (na // p) * w == E         # 32-byte row segments, E values
    n_tiles = nr // w
    per = CLUSTER // p
    units = -(-n_tiles // per)
    seen_tiles, seen_slots = [], []
    for unit in range(units):
        for rank in range(CLUSTER):
            sub, c = rank // p, rank % p
            tile = unit * per + sub
            assert tile < n_tiles                         # no idle CTA in any cluster
            rank0 = rank - c
            assert 0 <= rank0 and rank0 + p <= CLUSTER    # peers inside the cluster
            assert all(0 <= rank0 + k < CLUSTER for k in range(p))
            seen_slots.append(tile * p + c)
            if c == 0:
                seen_tiles.append(tile)
    assert sorted(seen_tiles) == list(range(n_tiles))
    # partial-sum slots: the per-patch launch's CTA indices 0 .. n_tiles * p - 1
    assert sorted(seen_slots) == list(range(n_tiles * p))


@pytest.mark.parametrize("na,nr", list(itertools.product(SIZES, SIZES)))
def test_row_blocks(na, nr):
    wr = row_w(nr)
    assert wr * nr == 8192                                # one CTA holds 8192 values
    blocks = na // wr
    assert blocks * wr == na
    rows = sorted(blk * wr + r for blk in range(blocks) for r in range(wr))
    assert rows == list(range(na))
