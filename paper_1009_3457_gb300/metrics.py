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
