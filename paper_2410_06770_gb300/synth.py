"""Seeded synthetic inputs for xGETT: contraction signatures, strided layouts
and values.

This module holds no contraction arithmetic.  It only decides shapes,
increments, buffer offsets and the values stored in buffers, so both the CUDA
path and the CPU oracle can be fed the same inputs.

Conventions (thesis Sec. 5.4-5.7 and Sec. 6):
  * column-major, element-unit increments (the layout figures with increments
    [1, 3, 9] for a rank-3 tensor and [1, 5, 25] for a sub-tensor of a 5x5x5
    parent);
  * a pointer addresses the element whose coordinates are all zero; with a
    negative increment the other elements sit at lower addresses, so such a
    tensor's coordinate-zero element has a positive offset into its buffer;
  * PERM[p] is the output position of free index p, where free indices are A's
    non-contracted modes in ascending order followed by B's (Sec. 5.6).

Random contraction generation follows the parameters the thesis lists for its
generator (Sec. 7): minimum/maximum rank, minimum/maximum extent and the number
of contracted modes; it always produces a valid contraction.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional, Sequence, Tuple

import numpy as np

# A value no kernel produces by accident: C gaps must keep it bit for bit.
C_GAP_SENTINEL = -1234567.875


@dataclass
class Layout:
    """Logical extents + increments of one tensor inside a flat buffer."""
    ext: Tuple[int, ...]
    inc: Tuple[int, ...]
    off: int      # element offset of the coordinate-zero element in the buffer
    size: int     # buffer length in elements

    @property
    def rank(self) -> int:
        return len(self.ext)

    @property
    def numel(self) -> int:
        n = 1
        for e in self.ext:
            n *= e
        return n

    def positions(self) -> np.ndarray:
        """Buffer positions of all logical elements, first coordinate fastest."""
        return _positions_f(self.ext, self.inc, self.off)


def _positions_f(ext, inc, off) -> np.ndarray:
    if len(ext) == 0:
        return np.array([off], dtype=np.int64)
    grids = np.meshgrid(*[np.arange(e, dtype=np.int64) for e in ext], indexing="ij")
    pos = np.full(grids[0].shape, off, dtype=np.int64)
    for g, s in zip(grids, inc):
        pos = pos + g * s
    return pos.reshape(-1, order="F")


def colmajor_strides(ext: Sequence[int]) -> Tuple[int, ...]:
    s, out = 1, []
    for e in ext:
        out.append(s)
        s *= max(int(e), 1)
    return tuple(out)


def layout_contiguous(ext: Sequence[int]) -> Layout:
    ext = tuple(int(e) for e in ext)
    n = 1
    for e in ext:
        n *= e
    return Layout(ext, colmajor_strides(ext), 0, max(n, 1))


def layout_rowmajor(ext: Sequence[int]) -> Layout:
    ext = tuple(int(e) for e in ext)
    rev = colmajor_strides(ext[::-1])[::-1]
    n = 1
    for e in ext:
        n *= e
    return Layout(ext, tuple(rev), 0, max(n, 1))


def layout_explicit(ext: Sequence[int], inc: Sequence[int]) -> Layout:
    """Given increments (possibly negative/zero); buffer sized to the span."""
    ext = tuple(int(e) for e in ext)
    inc = tuple(int(s) for s in inc)
    lo = sum((e - 1) * s for e, s in zip(ext, inc) if s < 0 and e > 0)
    hi = sum((e - 1) * s for e, s in zip(ext, inc) if s > 0 and e > 0)
    return Layout(ext, inc, -lo, hi - lo + 1)


def layout_padded(ext: Sequence[int], rng: np.random.Generator, pad_lo=1, pad_hi=5,
                  negative: bool = False) -> Layout:
    """Sub-tensor of the same rank, randomly placed in a parent whose extents are
    pad_lo..pad_hi larger (thesis Sec. 7, "sub-tensor of same rank"); with
    negative=True every increment is negated (Sec. 7, "sub-tensor negative
    increment")."""
    ext = tuple(int(e) for e in ext)
    pads = [int(rng.integers(pad_lo, pad_hi + 1)) for _ in ext]
    parent = [e + p for e, p in zip(ext, pads)]
    strides = colmajor_strides(parent)
    size = 1
    for e in parent:
        size *= e
    if not negative:
        start = [int(rng.integers(0, p + 1)) for p in pads]
        off = sum(s * t for s, t in zip(start, strides))
        return Layout(ext, strides, off, size)
    # reversed traversal: coordinate 0 sits at the high end of the block
    start = [int(rng.integers(0, p + 1)) for p in pads]
    off = sum((t + e - 1) * s for t, e, s in zip(start, ext, strides))
    return Layout(ext, tuple(-s for s in strides), off, size)


def layout_negative(ext: Sequence[int]) -> Layout:
    """Dense tensor read backwards in memory (thesis Sec. 7, "negative increment")."""
    ext = tuple(int(e) for e in ext)
    strides = colmajor_strides(ext)
    n = 1
    for e in ext:
        n *= e
    off = sum((e - 1) * s for e, s in zip(ext, strides) if e > 0)
    return Layout(ext, tuple(-s for s in strides), off, max(n, 1))


def layout_lower_rank(ext: Sequence[int], rng: np.random.Generator) -> Layout:
    """Sub-tensor of a parent whose rank is 1..3 higher and whose extents are
    1..3 larger (thesis Sec. 7, "sub-tensor of lower rank")."""
    ext = tuple(int(e) for e in ext)
    extra = int(rng.integers(1, 4))
    prank = len(ext) + extra
    slots = sorted(rng.choice(prank, size=len(ext), replace=False).tolist())
    parent = [0] * prank
    start = [0] * prank
    for i, slot in enumerate(slots):
        grow = int(rng.integers(1, 4))
        parent[slot] = ext[i] + grow
        start[slot] = int(rng.integers(0, grow + 1))
    for slot in range(prank):
        if slot not in slots:
            parent[slot] = int(rng.integers(1, 4))
            start[slot] = int(rng.integers(0, parent[slot]))
    strides = colmajor_strides(parent)
    size = 1
    for e in parent:
        size *= e
    off = sum(t * s for t, s in zip(start, strides))
    return Layout(ext, tuple(strides[s] for s in slots), off, size)


LAYOUT_KINDS = ("contig", "rowmajor", "padded", "negative", "padded_negative", "lower_rank")


def make_layout(ext: Sequence[int], kind: str, rng: np.random.Generator) -> Layout:
    if kind == "contig":
        return layout_contiguous(ext)
    if kind == "rowmajor":
        return layout_rowmajor(ext)
    if kind == "padded":
        return layout_padded(ext, rng)
    if kind == "negative":
        return layout_negative(ext)
    if kind == "padded_negative":
        return layout_padded(ext, rng, negative=True)
    if kind == "lower_rank":
        return layout_lower_rank(ext, rng)
    raise ValueError(kind)


@dataclass
class Signature:
    """The index part of an xGETT call: ranks, extents, contracted pairs, PERM."""
    exta: Tuple[int, ...]
    extb: Tuple[int, ...]
    conta: Tuple[int, ...]
    contb: Tuple[int, ...]
    perm: Tuple[int, ...]

    @property
    def conts(self) -> int:
        return len(self.conta)

    @property
    def rank_c(self) -> int:
        return len(self.exta) + len(self.extb) - 2 * self.conts

    def free_modes(self) -> List[Tuple[int, int]]:
        """(tensor, mode) of free index p: A's free modes ascending, then B's."""
        fa = [(0, m) for m in range(len(self.exta)) if m not in self.conta]
        fb = [(1, m) for m in range(len(self.extb)) if m not in self.contb]
        return fa + fb

    def extc(self) -> Tuple[int, ...]:
        out = [0] * self.rank_c
        for p, (t, m) in enumerate(self.free_modes()):
            out[self.perm[p]] = (self.exta if t == 0 else self.extb)[m]
        return tuple(out)


def random_signature(rng: np.random.Generator, min_rank=1, max_rank=5, min_ext=1, max_ext=5,
                     conts: Optional[int] = None, min_conts=0, max_conts=4,
                     rank_a: Optional[int] = None, rank_b: Optional[int] = None,
                     equal_ext: Optional[int] = None, max_elems: Optional[int] = None) -> Signature:
    """Random valid contraction (thesis Sec. 7 generator parameters)."""
    for _ in range(1000):
        ra = rank_a if rank_a is not None else int(rng.integers(min_rank, max_rank + 1))
        rb = rank_b if rank_b is not None else int(rng.integers(min_rank, max_rank + 1))
        if conts is not None:
            k = conts
        else:
            k = int(rng.integers(min_conts, min(max_conts, ra, rb) + 1))
        if k > ra or k > rb:
            continue
        draw = (lambda: equal_ext) if equal_ext is not None else \
            (lambda: int(rng.integers(min_ext, max_ext + 1)))
        exta = [draw() for _ in range(ra)]
        extb = [draw() for _ in range(rb)]
        conta = [int(x) for x in rng.choice(ra, size=k, replace=False)] if k else []
        contb = [int(x) for x in rng.choice(rb, size=k, replace=False)] if k else []
        for ma, mb in zip(conta, contb):
            extb[mb] = exta[ma]
        nfree = ra + rb - 2 * k
        perm = [int(x) for x in rng.permutation(nfree)]
        sig = Signature(tuple(exta), tuple(extb), tuple(conta), tuple(contb), tuple(perm))
        if max_elems is not None:
            sizes = [int(np.prod(exta, dtype=np.int64)), int(np.prod(extb, dtype=np.int64)),
                     int(np.prod(sig.extc(), dtype=np.int64))]
            if max(sizes) > max_elems:
                continue
        return sig
    raise RuntimeError("could not draw a signature within the limits")


@dataclass
class Problem:
    """A full xGETT call: signature + three layouts + buffers (numpy, host)."""
    sig: Signature
    la: Layout
    lb: Layout
    lc: Layout
    A: np.ndarray
    B: np.ndarray
    C: np.ndarray
    name: str = ""
    meta: dict = field(default_factory=dict)

    def args(self):
        """The 14 xGETT index arguments (without pointers)."""
        s = self.sig
        return dict(RANKA=len(s.exta), EXTA=s.exta, INCA=self.la.inc,
                    RANKB=len(s.extb), EXTB=s.extb, INCB=self.lb.inc,
                    CONTS=s.conts, CONTA=s.conta, CONTB=s.contb, PERM=s.perm,
                    INCC=self.lc.inc)

    def copy(self) -> "Problem":
        return Problem(self.sig, self.la, self.lb, self.lc, self.A.copy(), self.B.copy(),
                       self.C.copy(), self.name, dict(self.meta))


def draw_values(rng: np.random.Generator, n: int, dist: str, dtype) -> np.ndarray:
    dtype = np.dtype(dtype)
    complex_ = dtype.kind == "c"

    def real(m):
        if dist == "uniform":
            return rng.uniform(-1.0, 1.0, m)
        if dist == "normal":
            return rng.standard_normal(m)
        if dist == "int":
            return rng.integers(-8, 9, m).astype(np.float64)
        if dist == "smallint":
            return rng.integers(-2, 3, m).astype(np.float64)
        if dist == "logu":
            # magnitudes log-uniform over [1e-8, 1e8], random signs
            mag = 10.0 ** rng.uniform(-8.0, 8.0, m)
            return np.where(rng.integers(0, 2, m) == 1, mag, -mag)
        if dist == "ones":
            return np.ones(m)
        if dist == "zeros":
            return np.zeros(m)
        raise ValueError(dist)

    v = real(n)
    if complex_:
        v = v + 1j * real(n)
    return v.astype(dtype)


def _dense_order(layout: Layout):
    """If the layout fills its buffer exactly (a permutation of a column-major
    layout, offset 0), the mode order from smallest to largest increment."""
    if layout.off != 0 or layout.size != max(layout.numel, 1) or layout.numel == 0:
        return None
    order = sorted(range(layout.rank), key=lambda i: layout.inc[i])
    s = 1
    for i in order:
        if layout.ext[i] > 1 and layout.inc[i] != s:
            return None
        s *= layout.ext[i]
    return order


def fill(layout: Layout, values: np.ndarray, dtype, gap) -> np.ndarray:
    """Buffer of layout.size with `values` scattered to the logical positions
    (first coordinate fastest) and `gap` everywhere else."""
    dtype = np.dtype(dtype)
    order = _dense_order(layout)
    if order is not None:
        t = np.asarray(values, dtype=dtype).reshape(layout.ext, order="F")
        return np.ascontiguousarray(t.transpose(order)).ravel(order="F") if layout.rank > 1 \
            else np.array(values, dtype=dtype).reshape(-1)
    buf = np.full(layout.size, gap, dtype=dtype)
    if layout.numel:
        buf[_positions_f(layout.ext, layout.inc, layout.off)] = values
    return buf


def gather(layout: Layout, buf: np.ndarray) -> np.ndarray:
    """Logical values (first coordinate fastest) read back from a buffer."""
    if layout.numel == 0:
        return np.zeros(0, dtype=buf.dtype)
    order = _dense_order(layout)
    if order is not None and layout.rank > 1:
        shape = [layout.ext[i] for i in order]
        t = buf.reshape(shape, order="F")
        inv = np.argsort(order)
        return t.transpose(inv).ravel(order="F")
    return buf[_positions_f(layout.ext, layout.inc, layout.off)]


def logical(layout: Layout, buf: np.ndarray) -> np.ndarray:
    """The tensor as an ndarray of shape ext (column-major logical order)."""
    return gather(layout, buf).reshape(layout.ext, order="F") if layout.rank else gather(layout, buf).reshape(())


def gap_mask(layout: Layout) -> np.ndarray:
    m = np.ones(layout.size, dtype=bool)
    if layout.numel:
        m[_positions_f(layout.ext, layout.inc, layout.off)] = False
    return m


def make_problem(sig: Signature, rng: np.random.Generator, dtype=np.float64, dist="uniform",
                 kinds=("contig", "contig", "contig"), c_dist="zeros", name="",
                 seeds: Optional[Tuple[int, int]] = None, layouts=None) -> Problem:
    """Problem with values drawn from `dist`; input gaps hold NaN, C gaps hold
    C_GAP_SENTINEL."""
    if layouts is None:
        la = make_layout(sig.exta, kinds[0], rng)
        lb = make_layout(sig.extb, kinds[1], rng)
        lc = make_layout(sig.extc(), kinds[2], rng)
    else:
        la, lb, lc = layouts
    ra = np.random.default_rng(seeds[0]) if seeds else rng
    rb = np.random.default_rng(seeds[1]) if seeds else rng
    nan = np.nan if np.dtype(dtype).kind != "c" else complex(np.nan, np.nan)
    A = fill(la, draw_values(ra, la.numel, dist, dtype), dtype, nan)
    B = fill(lb, draw_values(rb, lb.numel, dist, dtype), dtype, nan)
    C = fill(lc, draw_values(rng, lc.numel, c_dist, dtype), dtype, C_GAP_SENTINEL)
    return Problem(sig, la, lb, lc, A, B, C, name)


# --------------------------------------------------------------------------
# Thesis test families (Sec. 7).  Each returns a Problem; `dist` and `dtype`
# select the value distribution.
# --------------------------------------------------------------------------
THESIS_TESTS = (
    "basic", "commutativity", "nothing", "scalar", "permutations", "rank_zero", "rank_one",
    "square0", "square1", "square2", "cube0", "cube1", "cube2", "cube3",
    "hypercube0", "hypercube1", "hypercube2", "hypercube3", "hypercube4",
    "subtensor_same_rank", "negative_increment", "subtensor_negative", "subtensor_lower_rank",
)


def thesis_signature(name: str, rng: np.random.Generator) -> Tuple[Signature, Tuple[str, str, str]]:
    contig = ("contig", "contig", "contig")
    if name in ("basic", "commutativity", "permutations"):
        return random_signature(rng, 1, 5, 1, 5, min_conts=0, max_conts=4), contig
    if name == "nothing":
        return random_signature(rng, 1, 5, 1, 5, conts=0), contig
    if name == "scalar":
        r = int(rng.integers(1, 6))
        return random_signature(rng, rank_a=r, rank_b=r, conts=r, min_ext=1, max_ext=5), contig
    if name == "rank_zero":
        r = int(rng.integers(1, 6))
        if rng.integers(0, 2):
            return random_signature(rng, rank_a=r, rank_b=0, conts=0), contig
        return random_signature(rng, rank_a=0, rank_b=r, conts=0), contig
    if name == "rank_one":
        r = int(rng.integers(1, 6))
        k = int(rng.integers(0, 2))
        if rng.integers(0, 2):
            return random_signature(rng, rank_a=r, rank_b=1, conts=k), contig
        return random_signature(rng, rank_a=1, rank_b=r, conts=k), contig
    for base, rank in (("square", 2), ("cube", 3), ("hypercube", 4)):
        if name.startswith(base) and name[len(base):].isdigit():
            k = int(name[len(base):])
            e = int(rng.integers(1, 6))
            return random_signature(rng, rank_a=rank, rank_b=rank, conts=k, equal_ext=e), contig
    if name == "subtensor_same_rank":
        return random_signature(rng, 1, 5, 1, 5), ("padded",) * 3
    if name == "negative_increment":
        return random_signature(rng, 1, 5, 1, 5), ("negative",) * 3
    if name == "subtensor_negative":
        return random_signature(rng, 1, 5, 1, 5), ("padded_negative",) * 3
    if name == "subtensor_lower_rank":
        return random_signature(rng, 1, 5, 1, 5), ("lower_rank",) * 3
    raise ValueError(name)


def thesis_problem(name: str, seed: int, dtype=np.float64, dist="uniform", c_dist="zeros") -> Problem:
    rng = np.random.default_rng(seed)
    sig, kinds = thesis_signature(name, rng)
    return make_problem(sig, rng, dtype, dist, kinds, c_dist, name=f"{name}/{seed}")


def swapped(p: Problem) -> Problem:
    """Same inputs with A and B exchanged and PERM rotated so the output layout
    is unchanged (thesis Sec. 7, "commutativity")."""
    s = p.sig
    na = len(s.exta) - s.conts
    nb = len(s.extb) - s.conts
    perm = tuple(s.perm[na:]) + tuple(s.perm[:na])
    sig = Signature(s.extb, s.exta, s.contb, s.conta, perm)
    assert len(perm) == na + nb
    return Problem(sig, p.lb, p.la, p.lc, p.B.copy(), p.A.copy(), p.C.copy(), p.name + "/swapped")


def rotated_output(p: Problem, n: int, rng: np.random.Generator) -> Problem:
    """PERM shifted left n times (thesis Sec. 7, "permutations"): each free index
    moves to a new output position; C gets a fresh contiguous layout for the new
    extents."""
    s = p.sig
    r = len(s.perm)
    perm = tuple((q - n) % r for q in s.perm) if r else ()
    sig = Signature(s.exta, s.extb, s.conta, s.contb, perm)
    lc = layout_contiguous(sig.extc())
    C = fill(lc, np.zeros(lc.numel, dtype=p.C.dtype), p.C.dtype, C_GAP_SENTINEL)
    return Problem(sig, p.la, p.lb, lc, p.A.copy(), p.B.copy(), C, p.name + f"/rot{n}")


# --------------------------------------------------------------------------
# Named workloads (contractions shaped like the thesis's test cases, scaled up)
# --------------------------------------------------------------------------
def cfg_small_dgett(dist="uniform", dtype=np.float64) -> Problem:
    """A(a,b,c,d)=(32,24,16,20) with mode a at stride 2 (padded buffer), seed 0;
    B(d,e,b,f)=(20,28,24,12) contiguous, seed 1; contract A.b-B.b and A.d-B.d;
    output (e,a,f,c) contiguous."""
    sig = Signature((32, 24, 16, 20), (20, 28, 24, 12), (1, 3), (2, 0), (1, 3, 0, 2))
    la = layout_explicit(sig.exta, (2, 64, 1536, 24576))
    la = Layout(la.ext, la.inc, 0, 2 * 32 * 24 * 16 * 20)
    lb = layout_contiguous(sig.extb)
    lc = layout_contiguous(sig.extc())
    rng = np.random.default_rng(0)
    return make_problem(sig, rng, dtype, dist, c_dist="zeros", seeds=(0, 1),
                        layouts=(la, lb, lc), name="dgett_small_32x24x16x20")


def cfg_cc(variant="plain", dtype=np.float64, scale=128, small_ij=32) -> Problem:
    """C[a,b,i,j] += sum_{c,d} A[a,b,c,d] B[c,d,i,j], a..d = scale, i,j = small_ij,
    N(0,1) values (A seed 2, B seed 3).
    variant 'plain': column-major everything; 'perm': output (i,a,j,b);
    'transA': A row-major; 'perm_transA': both."""
    n, m = scale, small_ij
    exta = (n, n, n, n)
    extb = (n, n, m, m)
    perm = (1, 3, 0, 2) if "perm" in variant else (0, 1, 2, 3)
    sig = Signature(exta, extb, (2, 3), (0, 1), perm)
    la = layout_rowmajor(exta) if "transA" in variant else layout_contiguous(exta)
    lb = layout_contiguous(extb)
    lc = layout_contiguous(sig.extc())
    rng = np.random.default_rng(6)
    return make_problem(sig, rng, dtype, "normal", c_dist="zeros", seeds=(2, 3),
                        layouts=(la, lb, lc), name=f"cc_{variant}_{n}x{m}")


def cfg_stream(dtype=np.float64, a_ext=(256, 256, 64), b_ext=(64, 8), c_host=True) -> Problem:
    """Outer product (CONTS=0) of rank-3 A and rank-2 B, output (A modes, B modes),
    uniform[-1,1] values (A seed 4, B seed 5), C = 0.  With c_host=False the
    (large) zero C is not materialised on the host: Problem.C is a 1-element
    placeholder and meta["c_zero"] is set."""
    sig = Signature(tuple(a_ext), tuple(b_ext), (), (), tuple(range(len(a_ext) + len(b_ext))))
    la, lb = layout_contiguous(a_ext), layout_contiguous(b_ext)
    lc = layout_contiguous(sig.extc())
    if c_host:
        rng = np.random.default_rng(7)
        return make_problem(sig, rng, dtype, "uniform", c_dist="zeros", seeds=(4, 5),
                            layouts=(la, lb, lc), name="stream_outer")
    A = fill(la, draw_values(np.random.default_rng(4), la.numel, "uniform", dtype), dtype, np.nan)
    B = fill(lb, draw_values(np.random.default_rng(5), lb.numel, "uniform", dtype), dtype, np.nan)
    return Problem(sig, la, lb, lc, A, B, np.zeros(1, dtype=dtype), "stream_outer", {"c_zero": True})


def capped_signature(rng: np.random.Generator, ra: int, rb: int, k: int, min_ext: int, max_ext: int,
                     cap: int) -> Signature:
    """Random signature with ranks ra, rb and k contracted pairs, extents drawn
    U{min_ext..max_ext}; while |A|, |B| or |C| exceeds `cap` elements, the
    largest extent of the most oversized tensor is redrawn below its current
    value (contracted extents stay paired), so the draw always terminates."""
    exta = [int(rng.integers(min_ext, max_ext + 1)) for _ in range(ra)]
    extb = [int(rng.integers(min_ext, max_ext + 1)) for _ in range(rb)]
    conta = [int(x) for x in rng.choice(ra, size=k, replace=False)] if k else []
    contb = [int(x) for x in rng.choice(rb, size=k, replace=False)] if k else []
    for ma, mb in zip(conta, contb):
        extb[mb] = exta[ma]
    perm = [int(x) for x in rng.permutation(ra + rb - 2 * k)]
    pair_b = dict(zip(conta, contb))
    pair_a = dict(zip(contb, conta))
    while True:
        sig = Signature(tuple(exta), tuple(extb), tuple(conta), tuple(contb), tuple(perm))
        sizes = [int(np.prod(exta, dtype=np.int64)), int(np.prod(extb, dtype=np.int64)),
                 int(np.prod(sig.extc(), dtype=np.int64)) if sig.rank_c else 1]
        worst = int(np.argmax(sizes))
        if sizes[worst] <= cap:
            return sig
        if worst == 0:
            modes = [(exta[m], 0, m) for m in range(ra)]
        elif worst == 1:
            modes = [(extb[m], 1, m) for m in range(rb)]
        else:
            modes = [(exta[m], 0, m) for m in range(ra) if m not in conta] + \
                    [(extb[m], 1, m) for m in range(rb) if m not in contb]
        e, t, m = max(modes)
        if e <= min_ext:
            return sig  # cannot shrink further
        new = int(rng.integers(min_ext, e))
        if t == 0:
            exta[m] = new
            if m in pair_b:
                extb[pair_b[m]] = new
        else:
            extb[m] = new
            if m in pair_a:
                exta[pair_a[m]] = new


def batched_signatures(n=4096, seed=7, min_ext=2, max_ext=64, cap=1 << 18,
                       pad_frac=0.25) -> List[dict]:
    """Signatures for the batched workload: CONTS ~ U{0..3}, each rank ~
    U{max(2,CONTS)..5}, extents U{min_ext..max_ext}, random contracted pairs and
    output permutation, `pad_frac` of problems with padded strides on every
    tensor, input dtype fp32 or bf16 with probability 1/2; free extents are
    redrawn until |A|, |B|, |C| <= cap elements."""
    rng = np.random.default_rng(seed)
    out = []
    while len(out) < n:
        k = int(rng.integers(0, 4))
        ra = int(rng.integers(max(2, k), 6))
        rb = int(rng.integers(max(2, k), 6))
        sig = capped_signature(rng, ra, rb, k, min_ext, max_ext, cap)
        padded = bool(rng.random() < pad_frac)
        dtype = "bf16" if rng.integers(0, 2) else "f32"
        pads = None
        if padded:
            pads = tuple(tuple(int(rng.integers(1, 5)) for _ in ext)
                         for ext in (sig.exta, sig.extb, sig.extc()))
        out.append(dict(sig=sig, padded=padded, pads=pads, dtype=dtype,
                        value_seed=int(rng.integers(0, 2**31 - 1))))
    return out


def layout_with_pads(ext: Sequence[int], pads: Optional[Sequence[int]]) -> Layout:
    """Sub-tensor at the origin of a parent with extents ext + pads."""
    if pads is None:
        return layout_contiguous(ext)
    parent = [e + p for e, p in zip(ext, pads)]
    strides = colmajor_strides(parent)
    size = 1
    for e in parent:
        size *= e
    return Layout(tuple(int(e) for e in ext), strides, 0, max(size, 1))
