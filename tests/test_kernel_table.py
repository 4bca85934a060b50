"""Host-side checks of the kernel instantiation table (kernels.py): the keys
the library registers the kernels under are unique (the registry returns
the first match, so a duplicate would silently shadow a kernel), every tile
variant and every narrow last-column kernel has the default kernel of the
same stencil and degree beside it (the plan selects a degree on the default
tile first), and every radius fits the cells a lane holds (x neighbours
come from the adjacent lane only)."""
import re

from paper_2001_01473_gb300 import kernels

CELLS_PER_LANE = 4  # the default kernels' cells per lane (CELLS_PER_LANE in the CUDA sources)


def _key(expr):
    """(ndim, shape, radius, dtype, bT, post, tile, part) of one entry
    expression, derived as the entry functions derive their KernelKey."""
    m = re.fullmatch(r"(\w+)<(.*)>\((.*)\)", expr)
    assert m, expr
    name, targs, call = m.groups()
    a = [t.strip() for t in targs.split(",")]
    if name == "entry2d":
        shape, r, bt = a[0], int(a[1]), int(a[2])
        post = a[5] if len(a) > 5 else "POST_NONE"
        v = int(a[6]) if len(a) > 6 else CELLS_PER_LANE
        return (2, shape, r, call, bt, post, 0 if v == CELLS_PER_LANE else 32 * v, 0), v
    if name == "entry3d":
        shape, r, bt = a[0], int(a[1]), int(a[2])
        post = a[6] if len(a) > 6 else "POST_NONE"
        v = int(a[7]) if len(a) > 7 else CELLS_PER_LANE
        part = int(a[9]) if len(a) > 9 else 0
        tile = int(a[10]) if len(a) > 10 else 0
        if tile:
            assert tile == 32 * v and part == 0, expr
        return (3, shape, r, call, bt, post, tile, part), v
    if name == "entry_star3d":
        r, bt, _nw, v, _rw, part = (int(x) for x in a)
        tile = 32 * v if (part == 0 and v != CELLS_PER_LANE) else 0
        return (3, "SH_STAR", r, "DT_F32", bt, "POST_NONE", tile, part), v
    if name == "entry_box1":
        return (3, "SH_BOX", int(a[0]), call, 1, "POST_NONE", 0, 0), CELLS_PER_LANE
    raise AssertionError(f"unknown entry {name}")


def _keys():
    out = []
    for hdr, expr in kernels.instantiations():
        k, v = _key(expr)
        out.append((k, v, expr))
    return out


def test_keys_are_unique():
    seen = {}
    for k, _v, expr in _keys():
        assert k not in seen, f"{expr} and {seen[k]} register the same key {k}"
        seen[k] = expr


def test_variants_and_narrow_kernels_have_a_default_beside_them():
    keys = {k for k, _v, _e in _keys()}
    for k, _v, expr in _keys():
        ndim, shape, r, dt, bt, post, tile, part = k
        if tile or part:
            assert (ndim, shape, r, dt, bt, post, 0, 0) in keys, f"{expr}: no default kernel at bT={bt}"


def test_radius_fits_the_cells_of_a_lane():
    for k, v, expr in _keys():
        assert k[2] <= v, f"{expr}: radius {k[2]} > {v} cells per lane"


def test_every_default_stencil_starts_at_degree_one():
    # the remainder pass of a run (T mod bT steps) and T < bT need the small
    # degrees: every built stencil has its default kernel at bT = 1
    keys = {k for k, _v, _e in _keys()}
    stencils = {(k[0], k[1], k[2], k[3], k[5]) for k in keys if not k[6] and not k[7]}
    for ndim, shape, r, dt, post in stencils:
        assert (ndim, shape, r, dt, 1, post, 0, 0) in keys, (ndim, shape, r, dt, post)
