"""Work and traffic counts used to report throughput (pure Python, no arithmetic of the method).

paper_ops_per_translation(p): the operation count per M2L translation that the
paper's Tables m2ltesla / m2lfermi (Sec. 4.1.2) use.  The paper does not state
it; 28 p (p + 7) reproduces every OPS. cell of both tables from the
translations/s cell within 0.5 %.

m2l_flops_per_translation(p): real floating-point operations of one complex
p x p matrix-vector product (p^2 complex multiply-adds, 8 flops each) --
the algorithmic work of one translation by Eq. (M2Lmat).

m2l_bytes_per_box(p, elem): algorithmic HBM traffic of one box of one level:
read its ME once and write its LE once (2 p complex values).
"""


def paper_ops_per_translation(p: int) -> int:
    return 28 * p * (p + 7)


def m2l_flops_per_translation(p: int) -> int:
    return 8 * p * p


def m2l_bytes_per_box(p: int, elem_bytes: int = 4) -> int:
    return 2 * p * 2 * elem_bytes


def uniform_translations(level: int, periodic: bool = False) -> int:
    """Interaction-list entries of a uniform level: closed form (6n-8)^2-(3n-2)^2, n = 2^l."""
    if level < 2:
        return 0
    n = 1 << level
    if periodic:
        return 27 * n * n
    return (6 * n - 8) ** 2 - (3 * n - 2) ** 2


def fgt_translations(g: int, ncut: int) -> int:
    """Source-target box pairs of a 2^g x 2^g grid with Chebyshev distance <= ncut."""
    n = 1 << g
    per_axis = sum(min(n - 1, t + ncut) - max(0, t - ncut) + 1 for t in range(n))
    return per_axis * per_axis


def fgt_flops_per_box_separable(p: int, taps_x: int, taps_y: int) -> int:
    """Two 1-D passes of p x p by p x p real products: 2 p^3 flops per tap."""
    return 2 * p ** 3 * (taps_x + taps_y)


def fgt_h2p_flops_per_pair(p: int) -> int:
    """Eq. (hermite) for one target and one source box, as the bilinear form
    h(t1)^T A h(t2): p^2 + p multiply-adds (the Hermite functions themselves are
    not counted)."""
    return 2 * (p * p + p)


def fgt_h2p_pairs(g: int, ncut: int, target_counts, source_nonempty) -> int:
    """Target-source box pairs that Hermite evaluation on the 2^g grid works on:
    every target times the source boxes holding coefficients (non-empty boxes)
    within Chebyshev distance ncut of its box.  target_counts: targets per box
    (4^g, row-major); source_nonempty: bool per box."""
    import numpy as np

    n = 1 << g
    s = np.asarray(source_nonempty, dtype=np.int64).reshape(n, n)
    c = np.zeros((n + 1, n + 1), dtype=np.int64)  # 2-D prefix sums of the non-empty mask
    c[1:, 1:] = s.cumsum(0).cumsum(1)
    t = np.asarray(target_counts, dtype=np.int64).reshape(n, n)
    total = 0
    for ty in range(n):
        y0, y1 = max(0, ty - ncut), min(n - 1, ty + ncut) + 1
        for tx in range(n):
            if t[ty, tx]:
                x0, x1 = max(0, tx - ncut), min(n - 1, tx + ncut) + 1
                total += int(t[ty, tx]) * int(c[y1, x1] - c[y0, x1] - c[y1, x0] + c[y0, x0])
    return total


def fgt_h2p_tc_mma_flops(g: int, ncut: int, target_counts, products: int = 3, p: int = 16, rows: int = 128) -> int:
    """Tensor-core flops that the tensor-core Hermite evaluation issues: per claim of up to
    `rows` targets of a box, one [rows x p] x [p x (w p)] product per source row and precision
    product, w x h the box's clipped neighbourhood (every box evaluated, full M tiles)."""
    import numpy as np

    n = 1 << g
    t = np.asarray(target_counts, dtype=np.int64).reshape(n, n)
    total = 0
    for ty in range(n):
        h = min(n - 1, ty + ncut) - max(0, ty - ncut) + 1
        for tx in range(n):
            if t[ty, tx]:
                w = min(n - 1, tx + ncut) - max(0, tx - ncut) + 1
                tiles = -(-int(t[ty, tx]) // rows)
                total += tiles * h * 2 * rows * (w * p) * p
    return total * products


def p2p_pairs(level: int, target_counts, source_counts, self_pairs: int = 0) -> int:
    """(target, source) pairs of the near field at `level`: each target times the sources of
    its box and the adjacent boxes, less `self_pairs` (targets that are sources)."""
    import numpy as np

    n = 1 << level
    s = np.pad(np.asarray(source_counts, dtype=np.int64).reshape(n, n), 1)
    near = sum(s[1 + dy:1 + dy + n, 1 + dx:1 + dx + n] for dy in (-1, 0, 1) for dx in (-1, 0, 1))
    return int((np.asarray(target_counts, dtype=np.int64).reshape(n, n) * near).sum()) - int(self_pairs)


def m2l_tc_mma_flops(levels, p: int, products: int = 3) -> int:
    """Tensor-core flops the tensor-core M2L issues over the given uniform levels: per tile of
    8 x 32 parents, 32 operator blocks x (2p / 16) K steps x ceil(8p / 128) M tiles of
    M = 128, N = 256, K = 16 products, `products` per step (3 for the BF16 hi/lo split)."""
    mt = -(-8 * p // 128)
    tiles = 0
    for lv in levels:
        np_ = 1 << (lv - 1)
        tiles += -(-np_ // 8) * -(-np_ // 32)
    return tiles * 32 * (2 * p // 16) * mt * products * 2 * 128 * 256 * 16


def fgt_h2t_tc_mma_flops(g: int, ncut: int, products: int = 3) -> int:
    """Tensor-core flops the tensor-core H2T issues: per pass, 2^g lines x 2^g / 8 segments of
    M = 128 rows, and per source offset (2 n_cut + 1 of them) one N = 32 product (the hi and lo
    planes of H_d) and one N = 16 product with the split, or one N = 16 product without; K = 16."""
    segs = (1 << g) * ((1 << g) // 8)
    per_d = 2 * 128 * 16 * (32 + 16) if products == 3 else 2 * 128 * 16 * 16
    return 2 * segs * (2 * ncut + 1) * per_d
