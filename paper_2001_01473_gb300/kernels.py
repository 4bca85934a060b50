"""Table of the sweep-kernel instantiations compiled into the library.

Each entry is (ndim, shape, radius, bT range, storage type, mode, dtype tag).
The build step (build.py) turns every entry into small translation units so
that nvcc compiles them in parallel.  Degrees bT are bounded by the register
ring each kernel keeps (bT * (2R+1) rows of 4 cells per lane): the paper's
own tuning range is bT in [1, 16] for 2D and [1, 8] for 3D (Section 5.3),
and its best FP32 degrees are 10/10/7/5 (star R1-4) and 10/5 (box R1-2)
(Table 5).
"""

STAR, BOX = "SH_STAR", "SH_BOX"

KERNELS_2D = [
    # FP32 plain method
    (STAR, 1, range(1, 11), "float", "MODE_PLAIN", "DT_F32"),
    (STAR, 2, range(1, 9), "float", "MODE_PLAIN", "DT_F32"),
    (STAR, 3, range(1, 6), "float", "MODE_PLAIN", "DT_F32"),
    (STAR, 4, range(1, 5), "float", "MODE_PLAIN", "DT_F32"),
    (BOX, 1, range(1, 11), "float", "MODE_PLAIN", "DT_F32"),
    (BOX, 2, range(1, 7), "float", "MODE_PLAIN", "DT_F32"),
    # FP64 plain method (FP64 fma bound on GB300: small degrees suffice)
    (STAR, 1, range(1, 4), "double", "MODE_PLAIN", "DT_F64"),
    (STAR, 2, range(1, 4), "double", "MODE_PLAIN", "DT_F64"),
    (STAR, 3, range(1, 3), "double", "MODE_PLAIN", "DT_F64"),
    (STAR, 4, range(1, 3), "double", "MODE_PLAIN", "DT_F64"),
    (BOX, 1, range(1, 4), "double", "MODE_PLAIN", "DT_F64"),
    (BOX, 2, range(1, 4), "double", "MODE_PLAIN", "DT_F64"),
    # high-order box (radius 3-4): temporal blocking stops paying, bT 1-2
    (BOX, 3, range(1, 3), "float", "MODE_PLAIN", "DT_F32"),
    (BOX, 4, range(1, 2), "float", "MODE_PLAIN", "DT_F32"),
    (BOX, 3, range(1, 2), "double", "MODE_PLAIN", "DT_F64"),
    (BOX, 4, range(1, 2), "double", "MODE_PLAIN", "DT_F64"),
    # precision forms: binary16 storage, Dot2-compensated FP32
    (STAR, 1, range(1, 11), "__half", "MODE_PLAIN", "DT_F16S"),
    (BOX, 1, range(1, 11), "__half", "MODE_PLAIN", "DT_F16S"),
    (STAR, 1, range(1, 9), "float", "MODE_DOT2", "DT_F32C"),
    (BOX, 1, range(1, 7), "float", "MODE_DOT2", "DT_F32C"),
]

# Wider 2D tile variants: (shape, radius, bT range, storage, mode, dtype,
# cells per lane, CTAs per SM the registers are sized for; 0 = estimate).
# A lane of the default kernel owns 4 cells, so a warp tile is 128 cells
# wide and loses 2 bT R of them to the overlap; 6 cells per lane lose a
# smaller share at the degrees whose level rings still fit 3 CTAs per SM.
# (8 per lane would need a 260-element TMA row box, above the 256-element
# limit of one box.)  The tuner times them beside the default kernels.
KERNELS_2D_WIDE = [
    (STAR, 1, range(4, 7), "float", "MODE_PLAIN", "DT_F32", 6, 0),
    (STAR, 2, range(2, 4), "float", "MODE_PLAIN", "DT_F32", 6, 3),
    (STAR, 3, range(2, 3), "float", "MODE_PLAIN", "DT_F32", 6, 3),
    (BOX, 1, range(3, 6), "float", "MODE_PLAIN", "DT_F32", 6, 3),
]
# (Measured and not kept, no gain over the default width: the radius-4 star
# and radius-2 box at bT 2, binary16 storage for the radius-1 star and box.)
# the same for division-type stencils (both forms): (shape, radius, bT
# range, storage, dtype, cells per lane, CTAs per SM)
KERNELS_DIV_2D_WIDE = [
    (STAR, 1, range(4, 7), "float", "DT_F32", 6, 0),
]


# 3D: (shape, radius, bT range, storage, mode, dtype, warps per CTA).  A CTA
# tile is (2 * warps) rows by 128 cells; the register rings of the whole
# tile (tile cells x (2R+1) planes x bT levels) must fit in one SM's
# register file, which bounds the tile height for a given degree.
KERNELS_3D = [
    (STAR, 2, range(1, 2), "float", "MODE_PLAIN", "DT_F32", 16),
    (STAR, 3, range(1, 2), "float", "MODE_PLAIN", "DT_F32", 16),
    (STAR, 4, range(1, 2), "float", "MODE_PLAIN", "DT_F32", 16),
    (BOX, 1, range(1, 3), "float", "MODE_PLAIN", "DT_F32", 16),
    (BOX, 1, range(3, 4), "float", "MODE_PLAIN", "DT_F32", 12),
    (STAR, 1, range(1, 2), "double", "MODE_PLAIN", "DT_F64", 16),
    (STAR, 2, range(1, 2), "double", "MODE_PLAIN", "DT_F64", 12),
    (STAR, 3, range(1, 2), "double", "MODE_PLAIN", "DT_F64", 8),
    (STAR, 4, range(1, 2), "double", "MODE_PLAIN", "DT_F64", 8),
    (BOX, 1, range(1, 2), "double", "MODE_PLAIN", "DT_F64", 12),
    (STAR, 1, range(1, 4), "__half", "MODE_PLAIN", "DT_F16S", 16),
    (STAR, 1, range(1, 4), "float", "MODE_DOT2", "DT_F32C", 16),
]


# FP32 3D stars on the sweep with one CTA barrier per plane
# (sweep3d_star.cuh): (radius, bT range, warps per CTA, rows per warp).  Tiles
# are 128 cells wide and (warps x rows per warp) rows high; radius 1 and 2
# also get the narrow last-column instance (R cells per lane, same rows).
# The level rings take bT (2R+1) 4 RW registers per thread and the published
# planes bT (R+1) planes of shared memory, so the higher degrees and radii
# run on fewer, fatter threads (12 warps: 170 registers per thread, 8 warps:
# 255).  At bT = 1 the radius 2-4 stars measured faster on the
# per-level-exchange sweep (395 / 272 / 199 against 360 / 227 / 110 GCell/s
# on 512^3), which keeps those degrees.  The radius-4 star at bT 2 spills
# part of its rings (no tile of this shape holds them in registers) and is
# built for the tuner to time.
KERNELS_3D_STAR = [
    (1, range(1, 4), 16, 2),
    (1, range(4, 5), 12, 2),
    (2, range(2, 3), 12, 2),
    (2, range(3, 4), 8, 3),
    (3, range(2, 3), 8, 3),
    (4, range(2, 3), 12, 2),
]

# Tile variants of the same sweep for the tuner: (radius, bT range, warps per
# CTA, rows per warp, cells per lane).  A 64 x 64 tile (2 cells per lane, 4
# rows per warp) holds the same ring registers per thread as the 128 x 32
# default, loses fewer of its cells to the overlap at bT >= 2 (0.82 of the
# tile is stored at bT 3 against 0.77), and reads a y neighbour from shared
# memory for half of its rows instead of all of them, at the cost of twice
# the x shuffles per cell.  Keyed by the tile width (64).  (Measured and not
# kept: the radius-2 star at 64 x 48 and 64 x 32 cells, bT 2 and 3, which the
# tuner did not pick over the default tiles on 512^3.)
KERNELS_3D_STAR_NARROW = [
    (1, range(2, 4), 16, 4, 2),
    (1, range(4, 5), 12, 4, 2),
]


# 3D tile shape per stencil: (cells per lane V, rows per warp RW); the CTA
# tile is (NW * RW) rows x (32 * V) cells.  128 x 2 by default; the FP64
# radius-1 star uses 64-cell-wide tiles of 4 rows per warp, which waste
# fewer overlap cells on 512-wide grids (measured faster there; in FP32 the
# extra shuffles and row addressing cost more than the overlap saves).  The
# FP64 radius-3 star takes 3 rows per warp (24-row tiles instead of 16, of
# which 2R = 6 rows are overlap): 14.8 against 11.1 GCell/s on 512^3, with
# the rings still in registers (236 per thread); for radius 4 the same
# spills, and for the FP32 radius-3 star a 48-row tile (12 warps x 4 rows)
# spilled and measured slower (224 against 317).
def geom3d(shape, r, s):
    if s == "double" and shape == STAR and r == 3:
        return (4, 3)
    return (2, 4) if (s == "double" and shape == STAR and r == 1) else (4, 2)


# Cells per lane of the narrow kernel that a 3D kernel gets for a pass's
# ragged last tile column (0: none).  With 128-cell tiles a 512-wide grid is
# 4 x (128 - 2 bT R) columns plus a remainder of a few dozen, which would
# otherwise take a fifth, mostly idle, full tile (FP64 radius-1 star:
# 64-cell tiles, 8 columns plus a remainder).  A lane's x neighbours must
# sit in the adjacent lanes, so the narrow kernel has R cells per lane:
# 32 or 64 cells wide for radius 1 or 2.  (A 96-cell kernel for radius 3
# measured slower than the full fifth tile: the narrow launch runs after the
# main one, and at 3 cells per lane it saves too little to pay for its own
# partial wave; radius 4 would need the full width.)
def tail3d(shape, r, s, mode):
    return r if r <= 2 and shape == STAR or r == 1 else 0


# One-level 3D box sweeps for radius 2-4 (sweep3d_box1.cuh): (radius, storage
# type, dtype tag, warps per CTA, rows per warp).  Each runs at bT = 1.
KERNELS_3D_BOX1 = [
    (2, "float", "DT_F32", 16, 2),
    (3, "float", "DT_F32", 12, 2),
    (4, "float", "DT_F32", 12, 2),
    (2, "double", "DT_F64", 16, 1),
    (3, "double", "DT_F64", 16, 1),
    (4, "double", "DT_F64", 16, 1),
]


# Division-type stencils (Table 4: j2d5pt = star2d R1, j2d9pt = star2d R2,
# j2d9pt-gol = box2d R1, j3d27pt = box3d R1, each divided by a constant every
# step), in both forms of the division: (shape, radius, bT range, storage
# type, dtype tag) and, in 3D, warps per CTA.
POSTS = ("POST_DIV", "POST_MUL")
KERNELS_DIV_2D = [
    (STAR, 1, range(1, 11), "float", "DT_F32"),
    (STAR, 2, range(1, 6), "float", "DT_F32"),
    (BOX, 1, range(1, 7), "float", "DT_F32"),
    (STAR, 1, range(1, 3), "double", "DT_F64"),
    (STAR, 2, range(1, 3), "double", "DT_F64"),
    (BOX, 1, range(1, 3), "double", "DT_F64"),
]
KERNELS_DIV_3D = [
    (BOX, 1, range(1, 3), "float", "DT_F32", 16),
    (BOX, 1, range(3, 4), "float", "DT_F32", 12),
    (BOX, 1, range(1, 2), "double", "DT_F64", 12),
]

# Tile variants of the per-level-exchange 3D sweep, timed by the tuner beside
# the default tile of the same stencil and degree: (shape, radius, bT range,
# storage, mode, dtype, warps per CTA, cells per lane, rows per warp,
# division forms).  64 x 64 tiles for the radius-1 box: the same registers per thread
# as the default 128 x 32 tile and a smaller share of overlap cells at
# bT >= 2.  (Its division forms were measured and not kept: the tuner kept
# the default tile for j3d27pt on 512^3.)
KERNELS_3D_VARIANTS = [
    (BOX, 1, range(1, 3), "float", "MODE_PLAIN", "DT_F32", 16, 2, 4, ("POST_NONE",)),
    (BOX, 1, range(3, 4), "float", "MODE_PLAIN", "DT_F32", 12, 2, 4, ("POST_NONE",)),
    (STAR, 2, range(1, 2), "double", "MODE_PLAIN", "DT_F64", 12, 2, 4, ("POST_NONE",)),
    (STAR, 1, range(1, 4), "float", "MODE_DOT2", "DT_F32C", 16, 2, 4, ("POST_NONE",)),
    (STAR, 1, range(1, 4), "__half", "MODE_PLAIN", "DT_F16S", 16, 2, 4, ("POST_NONE",)),
]


def instantiations():
    """Yield (header, entry expression) for every kernel instantiation."""
    for shape, r, bts, s, mode, dt in KERNELS_2D:
        for bt in bts:
            yield "sweep2d.cuh", f"entry2d<{shape}, {r}, {bt}, {s}, {mode}>({dt})"
    for shape, r, bts, s, mode, dt, v, occ in KERNELS_2D_WIDE:
        for bt in bts:
            yield "sweep2d.cuh", f"entry2d<{shape}, {r}, {bt}, {s}, {mode}, POST_NONE, {v}, {occ}>({dt})"
    for shape, r, bts, s, mode, dt, nw in KERNELS_3D:
        v, rw = geom3d(shape, r, s)
        for bt in bts:
            yield "sweep3d.cuh", f"entry3d<{shape}, {r}, {bt}, {s}, {mode}, {nw}, POST_NONE, {v}, {rw}>({dt})"
            tv = tail3d(shape, r, s, mode)
            if tv and tv < v:
                yield "sweep3d.cuh", f"entry3d<{shape}, {r}, {bt}, {s}, {mode}, {nw}, POST_NONE, {tv}, {rw}, 1>({dt})"
    for r, bts, nw, rw in KERNELS_3D_STAR:
        for bt in bts:
            yield "sweep3d_star.cuh", f"entry_star3d<{r}, {bt}, {nw}, 4, {rw}, 0>()"
            tv = tail3d(STAR, r, "float", "MODE_PLAIN")
            if tv and tv < 4:
                yield "sweep3d_star.cuh", f"entry_star3d<{r}, {bt}, {nw}, {tv}, {rw}, 1>()"
    for r, bts, nw, rw, v in KERNELS_3D_STAR_NARROW:
        for bt in bts:
            yield "sweep3d_star.cuh", f"entry_star3d<{r}, {bt}, {nw}, {v}, {rw}, 0>()"
    for r, s, dt, nw, rw in KERNELS_3D_BOX1:
        yield "sweep3d_box1.cuh", f"entry_box1<{r}, {s}, {nw}, {rw}>({dt})"
    for shape, r, bts, s, mode, dt, nw, v, rw, posts in KERNELS_3D_VARIANTS:
        for post in posts:
            for bt in bts:
                yield "sweep3d.cuh", (f"entry3d<{shape}, {r}, {bt}, {s}, {mode}, {nw}, {post}, {v}, {rw}, 0, "
                                      f"{32 * v}>({dt})")
    for post in POSTS:
        for shape, r, bts, s, dt in KERNELS_DIV_2D:
            for bt in bts:
                yield "sweep2d.cuh", f"entry2d<{shape}, {r}, {bt}, {s}, MODE_PLAIN, {post}>({dt})"
        for shape, r, bts, s, dt, v, occ in KERNELS_DIV_2D_WIDE:
            for bt in bts:
                yield "sweep2d.cuh", f"entry2d<{shape}, {r}, {bt}, {s}, MODE_PLAIN, {post}, {v}, {occ}>({dt})"
        for shape, r, bts, s, dt, nw in KERNELS_DIV_3D:
            v, rw = geom3d(shape, r, s)
            for bt in bts:
                yield "sweep3d.cuh", f"entry3d<{shape}, {r}, {bt}, {s}, MODE_PLAIN, {nw}, {post}, {v}, {rw}>({dt})"
                tv = tail3d(shape, r, s, "MODE_PLAIN")
                if tv and tv < v:
                    yield "sweep3d.cuh", (f"entry3d<{shape}, {r}, {bt}, {s}, MODE_PLAIN, {nw}, {post}, {tv}, {rw}, 1>"
                                          f"({dt})")
