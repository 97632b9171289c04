"""Host check of the persistent column pass's index arithmetic (colp_pass.cuh), for every
instantiated configuration, before any of it runs on a GPU: the landing-buffer reads,
the tensor-copy boxes and their coordinates (inside the array, innermost coordinate a
multiple of 16 bytes), the cross-CTA pushes and reads of the exchange buffer, the
selection histogram, the column-order mask words, the output rows, the shared-memory
size, and that the slots each thread reads and the pushes each CTA receives are a
permutation (every element written once and read once).  Mirrors the kernel's formulas;
no GPU needed."""
import pytest

# (N, P, E) of CSAR_COLP_CONFIGS
CONFIGS = [(8192, 8, 4096), (8192, 16, 4096), (4096, 4, 4096), (2048, 2, 4096), (1024, 1, 4096)]
TW = 192            # twiddle table entries
HIST_BINS = 4096
SMEM_LIMIT = 227 * 1024


def cfg(n, p, e):
    w = max(1, min(16, e * p // n))
    q = n // p
    r = 16                       # col_regs
    qr = q // r
    nt = qr * w
    return dict(W=w, Q=q, R=r, QR=qr, NT=nt, RP=r // p, QB=q // p, BR=min(q // p, 256))


def at4(q, w_, wc, n_):
    f = n_ * w_ + wc             # column layout, one pad slot every 16 elements
    return f + (f >> 4)


@pytest.mark.parametrize("n,p,e", CONFIGS)
def test_persistent_column_pass_indexing(n, p, e):
    c = cfg(n, p, e)
    W, Q, R, QR, NT, RP, QB, BR = (c[k] for k in ("W", "Q", "R", "QR", "NT", "RP", "QB", "BR"))
    assert QB % BR == 0 and BR <= 256 and W * 8 % 16 == 0
    smem_x = Q * W + Q * W // 16
    smem = e * 8 + smem_x * 8 + TW * 8 + 32 * 4 + 6 * 8 + NT * 4
    assert smem <= SMEM_LIMIT
    assert HIST_BINS * 4 <= smem_x * 8
    nr = 64 * W
    n_tiles = nr // W
    for tile in (0, n_tiles - 1):
        # boxes: x = tile W (multiple of 16 bytes), rows inside [0, N)
        x = tile * W
        assert x * 8 % 16 == 0 and x + W <= nr
        for cc in range(p):
            cover = set()
            for n1 in range(p):
                for b in range(QB // BR):
                    y = n1 * Q + cc * QB + b * BR
                    assert 0 <= y and y + BR <= n
                    dst = (n1 * QB + b * BR) * W
                    assert dst * 8 % 16 == 0 and dst + BR * W <= e
                    cover.update(range(dst, dst + BR * W))
            assert cover == set(range(e))
    # landing reads: thread (t, w), slot i P + n1 -> element (n1 QB + t + QR i) W + w, a
    # permutation of the landing buffer
    reads = [(n1 * QB + t + QR * i) * W + w for t in range(QR) for w in range(W)
             for i in range(RP) for n1 in range(p)]
    assert sorted(reads) == list(range(e))
    if p > 1:
        # blocked-input pushes: CTA cc, thread (t, w), i -> element n2 = cc QB + t + QR i of
        # every CTA k1: each CTA receives every (w, n2) exactly once
        got = sorted(at4(Q, W, w, cc * QB + t + QR * i)
                     for cc in range(p) for t in range(QR) for w in range(W) for i in range(RP))
        want = sorted(at4(Q, W, w, m) for w in range(W) for m in range(Q))
        assert got == want and max(got) < smem_x
        # strided-input pushes of the residue pass: CTA cc, slot s -> CTA s // RP, element
        # cc QB + t + QR (s % RP); each CTA receives every element once
        recv = {}
        for cc in range(p):
            for t in range(QR):
                for w in range(W):
                    for s in range(R):
                        dst = s // RP
                        recv.setdefault(dst, []).append(at4(Q, W, w, cc * QB + t + QR * (s % RP)))
        for dst, lst in recv.items():
            assert sorted(lst) == want, dst
        # the length-P DFT reads n1 QB + k2l, k2l = t + QR i
        rd = sorted(at4(Q, W, w, n1 * QB + t + QR * i)
                    for t in range(QR) for w in range(W) for i in range(RP) for n1 in range(p))
        assert rd == want
        # output rows of the residue pass: (cc QB + t + QR i) + k1 Q, all of [0, N) once
        rows = sorted(cc * QB + t + QR * i + k1 * Q
                      for cc in range(p) for t in range(QR) for i in range(RP) for k1 in range(p))
        assert rows == list(range(n))
    # strided output rows of the forward / inverse passes: cc + P (t + s QR)
    rows = sorted(cc + p * (t + s * QR) for cc in range(p) for t in range(QR) for s in range(R))
    assert rows == list(range(n))
    # column-order mask words: ((col P + cc) QR + t) < nr (N / R)
    assert ((nr - 1) * p + (p - 1)) * QR + (QR - 1) < nr * (n // R)
