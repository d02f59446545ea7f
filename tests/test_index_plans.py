"""CPU replays of the frame kernel's index plans (no GPU).

The index arithmetic of the CUDA kernels is restated here for whole ranges of
sizes, and every replay checks that each load and store stays inside its
buffer with the alignment of its vector width, and that the work partitions
cover every element exactly once.  The formulas follow prost_frame.cuh
(FrameTiles, the residual pass's items, the update pass's items,
reduce_rows), prost_stage.cuh (the streaming form's 16-byte copies of a
step into its stage), prost_api.cu (the frame grid and the partial-row stride) and
prost_window.cu (the U-step's reductions); the constants are read from those
sources, so a change of tile size or reduction shape is replayed too."""

import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1302_2073_gb300", "csrc")


def _src(name):
    with open(os.path.join(CSRC, name)) as f:
        return f.read()


def _const(text, pattern):
    m = re.search(pattern, text)
    assert m, pattern
    return int(m.group(1))


DEVICE_H, FRAME_CUH, API_CU, WINDOW_CU = (_src(n) for n in ("prost_device.h", "prost_frame.cuh", "prost_api.cu",
                                                          "prost_window.cu"))
TILE_P = _const(DEVICE_H, r"constexpr int TILE_P = (\d+);")
RW = _const(FRAME_CUH, r"static constexpr int RW = (\d+);")
RED_ROWS = _const(DEVICE_H, r"constexpr int RED_ROWS = (\d+);")
RED_SCR = _const(DEVICE_H, r"constexpr int RED_SCR = (\d+);")
assert "constexpr int max_frame_grid(int nv) { return RED_SCR / nv * RED_ROWS; }" in DEVICE_H
assert "int col_stride(int grid) { return (grid + 3) / 4 * 4; }" in API_CU
WT = _const(WINDOW_CU, r"constexpr int WT = (\d+);")
KMAXW = _const(WINDOW_CU, r"constexpr int KMAXW = (\d+);")
IPT = TILE_P // RW
SMS = 152

# the rules restated below, as they read in the sources
assert "static constexpr int THREADS = STREAM && sizeof(UT) == 4 ? 256 : 512;" in FRAME_CUH
KREG = _const(DEVICE_H, r"constexpr int KREG = (\d+);")
assert KREG == 10 and "static constexpr bool STREAM = K > KREG;" in FRAME_CUH
assert "return (size_t)k + (size_t)k * (k + 1) / 2 + 3;" in API_CU
assert "r0 = (int)(NT * b / G);" in FRAME_CUH and "u0 = (int)((long long)prm.npt * b / G);" in FRAME_CUH


def threads(k, bf16):
    return 256 if (k >= 11 and not bf16) else 512


def partial_row(k):
    return k + k * (k + 1) // 2 + 3


def npt_of(P):
    return (P + TILE_P - 1) // TILE_P


def frame_grid(P, sms=SMS, occ=1, k=1):
    """The frame kernel's grid: one CTA per SM, at most one per pixel tile,
    at most what the reduction's scratch takes."""
    return max(1, min(occ * sms, npt_of(P), RED_SCR // partial_row(k) * RED_ROWS))


def frame_tiles(C, npt, G, b):
    """(r0, nres, u0, nupt) of CTA b: its residual-pass tiles (over all
    channel planes) and its update-pass pixel tiles."""
    NT = C * npt
    r0 = NT * b // G
    u0 = npt * b // G
    return r0, NT * (b + 1) // G - r0, u0, npt * (b + 1) // G - u0


SHAPES = [(1, 1), (7, 1), (223, 1), (224, 1), (225, 3), (37 * 29, 3), (160 * 120, 1), (160 * 120, 3),
          (320 * 240, 1), (640 * 480, 3), (1280 * 720, 1), (1920 * 1080, 3)]


def _grids(P):
    npt = npt_of(P)
    return sorted({g for g in (1, 2, 7, 19, frame_grid(P), npt) if 1 <= g <= npt})


@pytest.mark.parametrize("P,C", SHAPES)
def test_frame_tiles_partition_the_planes(P, C):
    npt = npt_of(P)
    for G in _grids(P):
        res_cover = np.zeros(C * npt, np.int64)
        upd_cover = np.zeros(npt, np.int64)
        for b in range(G):
            r0, nres, u0, nupt = frame_tiles(C, npt, G, b)
            assert nres >= 1 and nupt >= 1, (P, C, G, b)
            res_cover[r0:r0 + nres] += 1
            upd_cover[u0:u0 + nupt] += 1
        assert (res_cover == 1).all() and (upd_cover == 1).all(), (P, C, G)


@pytest.mark.parametrize("P,C", SHAPES)
@pytest.mark.parametrize("k", [1, 10])
def test_residual_pass_loads_stay_in_bounds_and_aligned(P, C, k):
    """Items of the register form: tile ti, pair rp; U pair loads at
    ti*k*TP + rp*RW + j*TP, the frame's pair (or single) load at c*pitch + p,
    the labels' pair load at p (the label plane is padded)."""
    npt = npt_of(P)
    Pp = npt * TILE_P
    ti, rp = np.meshgrid(np.arange(C * npt, dtype=np.int64), np.arange(IPT, dtype=np.int64), indexing="ij")
    ti, rp = ti.ravel(), rp.ravel()
    c = ti // npt
    p = (ti - c * npt) * TILE_P + rp * RW
    nvalid = np.minimum(P - p, RW)
    # every entry of every plane is read exactly once, padding entries never
    q = np.concatenate([c * P + p + r for r in range(RW)])
    valid = np.concatenate([nvalid > r for r in range(RW)])
    counts = np.bincount(q[valid], minlength=C * P)
    assert counts.size == C * P and (counts == 1).all()
    # the subspace: pair loads inside C*npt*k*TP entries, at even offsets
    for j in (0, k - 1):
        off = ti * k * TILE_P + rp * RW + j * TILE_P
        assert off.min() >= 0 and (off + RW - 1).max() < C * npt * k * TILE_P
        assert (off % RW == 0).all()
    # the frame, direct (pitch P, only when planes are 16-byte multiples) or staged (pitch Pp)
    for eb in (1, 4):
        pitches = [Pp] + ([P] if (P * eb) % 16 == 0 else [])
        for pitch in pitches:
            base = c * pitch + p
            pair = nvalid == RW
            assert ((base[pair] * eb) % (RW * eb) == 0).all()
            assert (base[pair] + RW - 1).max(initial=0) < C * pitch
            one = (nvalid >= 1) & ~pair
            assert base[one].max(initial=0) < C * pitch
    # the labels: a pair load at p in a plane of Pp bytes
    assert (p + RW - 1).max() < Pp and (p % RW == 0).all()


@pytest.mark.parametrize("P,C", SHAPES)
def test_update_pass_touches_every_row_once(P, C):
    """Items of the update pass: a CTA's pixel tiles, one pixel per item, its
    channels in turn; the row of pixel p in plane c is written once, labels
    once per pixel."""
    k = 3
    npt = npt_of(P)
    Pp = npt * TILE_P
    G = frame_grid(P)
    row_writes = np.zeros(C * npt * k * TILE_P, np.int64)
    label_writes = np.zeros(Pp, np.int64)
    for b in range(G):
        _, _, u0, nupt = frame_tiles(C, npt, G, b)
        it = np.arange(nupt * TILE_P, dtype=np.int64)
        pt = u0 + it // TILE_P
        r0 = it % TILE_P
        p = pt * TILE_P + r0
        for ch in range(C):
            for j in range(k):
                np.add.at(row_writes, (ch * npt + pt) * k * TILE_P + r0 + j * TILE_P, 1)
            frame_off = ch * P + p[p < P]           # frame reads, direct pitch
            assert frame_off.size == 0 or frame_off.max() < C * P
        np.add.at(label_writes, p, 1)
    assert (row_writes == 1).all()
    assert (label_writes == 1).all()


def _reduce_plan(nrows, nv, ncons):
    """reduce_rows: the groups, the units each thread sums, and the rows each
    unit reads."""
    ng = max(-(-nrows // RED_ROWS), ncons // nv)
    ng = max(1, min(ng, min(nrows, RED_SCR // nv)))
    nu = ng * nv
    by_thread = []
    for t in range(ncons):
        mine = []
        if nu <= ncons:
            if t < nu:
                mine.append(t)
        else:
            u0 = t
            while u0 < nu:
                u1 = u0 + ncons
                mine.append(u0)
                if u1 < nu:
                    mine.append(u1)
                u0 += 2 * ncons
        by_thread.append(mine)
    return ng, nu, by_thread


def _reduce_cases():
    cases = set()
    for k in range(1, 17):
        for bf16 in (False, True):
            nt = threads(k, bf16)
            stride = partial_row(k)
            for nv in (k + k * (k + 1) // 2 + 3, k + 3, k * (k + 1) // 2 + 1):
                cases.add((nt, stride, nv))
    for k in range(1, KMAXW + 1):
        for nv in (k * k, k * (k + 1) // 2):
            cases.add((WT, KMAXW * KMAXW, nv))
    return sorted(cases)


@pytest.mark.parametrize("ncons,stride,nv", _reduce_cases())
def test_reduce_rows_plan_sums_every_value_of_every_row_once(ncons, stride, nv):
    assert nv <= stride
    for nrows in (1, 2, 23, 24, 25, 76, 151, 152, 304, 1024):
        ng, nu, by_thread = _reduce_plan(nrows, nv, ncons)
        assert nu <= RED_SCR                                  # scratch of the group sums
        units = [u for mine in by_thread for u in mine]
        assert sorted(units) == list(range(nu))               # each unit by one thread
        seen = np.zeros((nrows, nv), np.int64)
        for u in range(nu):
            g, c = divmod(u, nv)
            rows = np.arange(g, nrows, ng)
            off = rows * stride + c
            assert off.size == 0 or off.max() < nrows * stride
            seen[rows, c] += 1
        assert (seen == 1).all()
        # the final sums read scr[g*nv + c], g < ng: exactly the units written
        assert sorted(g * nv + c for c in range(nv) for g in range(ng)) == list(range(nu))


def _cols_cases():
    cases = set()
    for k in range(1, 17):
        for bf16 in (False, True):
            for nv in (k + k * (k + 1) // 2 + 3, k + 3, k * (k + 1) // 2 + 1, 1):
                cases.add((threads(k, bf16), partial_row(k), nv))
    return sorted(cases)


@pytest.mark.parametrize("ncons,nvmax,nv", _cols_cases())
def test_reduce_cols_plan_sums_every_value_of_every_cta_once(ncons, nvmax, nv):
    """reduce_cols: value c of CTA b at c * cstride + b, cstride = the grid
    rounded up to 4; unit u = c nq + q sums rows [q RED_ROWS, (q+1) RED_ROWS)
    with 16-byte loads, each issued only where it starts below nrows."""
    assert RED_ROWS % 4 == 0
    for nrows in sorted({1, 2, 3, 4, 5, 23, 24, 25, 76, 151, 152, SMS, RED_SCR // nvmax * RED_ROWS}):
        if nrows > RED_SCR // nvmax * RED_ROWS:
            continue
        cs = (nrows + 3) // 4 * 4
        nq = -(-nrows // RED_ROWS)
        nu = nq * nv
        assert nu <= RED_SCR                                   # the unit sums fit the scratch
        buf = nvmax * cs                                       # one buffer of the frame kernel
        seen = np.zeros((nv, nrows), np.int64)
        for u in range(nu):
            c, q = divmod(u, nq)
            r0 = q * RED_ROWS
            for i in range(RED_ROWS // 4):
                r = r0 + 4 * i
                if r >= nrows:
                    continue
                off = c * cs + r
                assert off % 4 == 0 and off + 3 < (c + 1) * cs <= buf  # inside the value's entries
                for j in range(4):
                    if r + j < nrows:
                        seen[c, r + j] += 1
        assert (seen == 1).all()
        # the per-value sums read scr[c nq + q], exactly the units written
        assert sorted(c * nq + q for c in range(nv) for q in range(nq)) == list(range(nu))


# ---- the streaming form's staging plan (prost_stage.cuh) -----------------------

STAGE_CUH = _src("prost_stage.cuh")
STG_ROWS = _const(STAGE_CUH, r"constexpr int STG_ROWS = (\d+);")
TC_CS = _const(STAGE_CUH, r"static constexpr int CS = TC \? (\d+) : STG_ROWS;")
assert "static constexpr int UCOL = TC ? 16 : K;" in STAGE_CUH
assert "uoff = (lane / S::CPC) * TILE_P + (lane % S::CPC) * RPC;" in STAGE_CUH
assert "soff = (lane / S::CPC) * S::CS * (int)sizeof(UT) + 16 * (lane % S::CPC);" in STAGE_CUH


def stage_cfg(k, fsize, usize):
    tc = usize == 2
    cs = TC_CS if tc else STG_ROWS
    ucol = 16 if tc else k
    ub = ucol * cs * usize
    f_off = ub
    l_off = f_off + STG_ROWS * fsize
    stage_b = (l_off + STG_ROWS + 127) // 128 * 128
    cpc = STG_ROWS * usize // 16
    ncu = k * cpc
    ncf = STG_ROWS * fsize // 16
    ncl = STG_ROWS // 16
    return dict(cs=cs, ub=ub, f_off=f_off, l_off=l_off, stage_b=stage_b, cpc=cpc, ncu=ncu, ncf=ncf, ncl=ncl,
                nch=ncu + ncf + ncl)


def lane_copies(k, fsize, usize, lane):
    """(kind, stage byte offset, source offset) of every 16-byte copy lane
    issues for one step: kind 'u' (source in elements from the tile's block at
    row rs), 'f' (elements from the step's first frame entry), 'l' (bytes
    from its first label)."""
    S = stage_cfg(k, fsize, usize)
    nqu = S["ncu"] // 32
    tr = (S["nch"] - 32 * nqu + 31) // 32
    qcol = 32 // S["cpc"]
    rpc = 16 // usize
    qb = qcol * S["cs"] * usize
    uoff = (lane // S["cpc"]) * TILE_P + (lane % S["cpc"]) * rpc
    soff = (lane // S["cpc"]) * S["cs"] * usize + 16 * (lane % S["cpc"])
    out = [("u", soff + q * qb, uoff + q * qcol * TILE_P) for q in range(nqu)]
    for r in range(tr):
        ch = 32 * (nqu + r) + lane
        if ch < S["ncu"]:
            out.append(("u", soff + (nqu + r) * qb, uoff + (nqu + r) * qcol * TILE_P))
        elif ch < S["ncu"] + S["ncf"]:
            out.append(("f", S["f_off"] + 16 * (ch - S["ncu"]), (ch - S["ncu"]) * (16 // fsize)))
        elif ch < S["nch"]:
            out.append(("l", S["l_off"] + 16 * (ch - S["ncu"] - S["ncf"]), 16 * (ch - S["ncu"] - S["ncf"])))
    return S, out


@pytest.mark.parametrize("k", range(11, 17))
@pytest.mark.parametrize("fsize,usize", [(1, 4), (4, 4), (1, 2), (4, 2)])
def test_streaming_stage_copies_cover_the_step_once(k, fsize, usize):
    copies = [c for lane in range(32) for c in lane_copies(k, fsize, usize, lane)[1]]
    S = lane_copies(k, fsize, usize, 0)[0]
    dst = [d for _, d, _ in copies]
    assert len(dst) == len(set(dst))                                   # no stage byte written twice
    assert all(d % 16 == 0 and 0 <= d and d + 16 <= S["stage_b"] for d in dst)
    assert S["stage_b"] % 128 == 0
    # the subspace block: column j, row part q of the step at stage j*CS*s + 16 q,
    # read from element j*TP + q*(16/s) of the tile's block, every (j, q) once
    u = sorted((d, s) for kind, d, s in copies if kind == "u")
    want = sorted((j * S["cs"] * usize + 16 * q, j * TILE_P + q * (16 // usize))
                  for j in range(k) for q in range(S["cpc"]))
    assert u == want
    assert all(d + 16 <= S["ub"] for d, _ in u)
    # bfloat16: columns k .. 15 of the block are zeroed once per stage and no
    # copy lands there
    assert all(d + 16 <= k * S["cs"] * usize for d, _ in u)
    # the sources are 16-byte aligned: tile bases (k*TP elements apart) and
    # step starts (STG_ROWS rows) are, and so is every chunk offset
    assert (k * TILE_P * usize) % 16 == 0 and (STG_ROWS * usize) % 16 == 0
    assert all((s * usize) % 16 == 0 for _, s in u)
    # the frame entries and labels of the step, each slot once, in order
    f = sorted((d, s) for kind, d, s in copies if kind == "f")
    assert f == [(S["f_off"] + 16 * i, i * (16 // fsize)) for i in range(S["ncf"])]
    lab = sorted((d, s) for kind, d, s in copies if kind == "l")
    assert lab == [(S["l_off"] + 16 * i, 16 * i) for i in range(S["ncl"])]
    assert S["l_off"] + STG_ROWS <= S["stage_b"] and S["l_off"] % 16 == 0


@pytest.mark.parametrize("P", [37 * 29, 224, 1000, 1920 * 1080])
@pytest.mark.parametrize("fsize", [1, 4])
def test_streaming_frame_chunks_never_cross_the_plane_end(P, fsize):
    """A frame chunk is copied when its first entry is inside the plane
    (rs + offset < valid rows), else zero-filled.  On the direct pitch (planes
    are 16-byte multiples) a chunk that starts inside therefore ends inside;
    on the staged pitch it ends inside the padded plane."""
    per = 16 // fsize
    npt = npt_of(P)
    Pp = npt * TILE_P
    starts = np.arange(0, Pp, per, dtype=np.int64)       # chunk starts: tile, step and slot multiples
    inside = starts < P
    assert (starts[inside] + per <= Pp).all()
    if (P * fsize) % 16 == 0:
        assert (starts[inside] + per <= P).all()


# ---- the pre-processing resampler's footprints (prost_prepost.cu) --------------

PREPOST_CU = _src("prost_prepost.cu")
assert "lo = (int64_t)i * n_in;" in PREPOST_CU and "hi = lo + n_in;" in PREPOST_CU
assert "q0 = (int)(lo / n_out);" in PREPOST_CU
assert "q1 = (int)min((int64_t)n_in, (hi + n_out - 1) / n_out);" in PREPOST_CU
assert "return min(hi, (int64_t)(q + 1) * n_out) - max(lo, (int64_t)q * n_out);" in PREPOST_CU


def _pairs():
    rng = np.random.default_rng(0)
    fixed = [(640, 160), (480, 120), (1920, 160), (1080, 120), (1366, 160), (768, 120), (100, 37), (75, 29),
             (33, 40), (21, 30), (7, 3), (3, 8), (1, 5), (5, 1), (4096, 4095), (4095, 4096), (1, 1)]
    rand = [tuple(int(v) for v in rng.integers(1, 4097, size=2)) for _ in range(40)]
    return fixed + rand


@pytest.mark.parametrize("n_in,n_out", _pairs())
def test_resampling_footprints_stay_in_the_input_and_cover_it_exactly(n_in, n_out):
    """Output i reads input rows [floor(i n_in / n_out), min(n_in, ceil((i + 1)
    n_in / n_out))) with integer overlaps in units of 1 / n_out: never outside
    the input, never empty, every overlap positive, each output's overlaps
    adding up to n_in (weights summing to exactly one) and each input pixel's
    to n_out (its whole area used once)."""
    i = np.arange(n_out, dtype=np.int64)
    lo = i * n_in
    hi = lo + n_in
    q0 = lo // n_out
    q1 = np.minimum(n_in, (hi + n_out - 1) // n_out)
    assert q0.min() >= 0 and q1.max() <= n_in and (q1 > q0).all()
    used = np.zeros(n_in, np.int64)
    width = q1 - q0
    for w in np.unique(width):
        sel = np.nonzero(width == w)[0]
        q = q0[sel][:, None] + np.arange(w)[None, :]
        ov = np.minimum(hi[sel][:, None], (q + 1) * n_out) - np.maximum(lo[sel][:, None], q * n_out)
        assert (ov > 0).all()
        assert (ov.sum(axis=1) == n_in).all()
        np.add.at(used, q.ravel(), ov.ravel())
    assert (used == n_out).all()
    # the weights the kernel forms, ov as float32 (exact below 2^24)
    assert max(n_in, n_out) < 2 ** 24


# ---- the window kernel's shared memory (prost_window.cu) -----------------------

NMAXW = _const(WINDOW_CU, r"constexpr int NMAXW = (\d+);")
assert "float *Hs = Ys + K4 * a.n;" in WINDOW_CU
assert "float *Us = Hs + (GRAD ? WT * (a.n + 1) : 0); // WT x US" in WINDOW_CU
assert "w->smem_cost = (size_t)((k + 3) / 4 * 4) * n * sizeof(float);" in WINDOW_CU
assert "w->smem_grad = w->smem_cost + grad_floats * sizeof(float);" in WINDOW_CU


@pytest.mark.parametrize("k", range(1, KMAXW + 1))
def test_window_shared_memory_carve_up_fits_the_launch(k):
    """Ys (n x K4), then with gradients Hs (WT x (n + 1)) and Us (WT x US, k
    rounded up to even), at least WT x 8 floats after Ys: the carve-up ends
    inside the dynamic shared memory each launch asks for, which stays inside
    the 227 KB a CTA may have; Us starts 8-byte aligned for its pair loads."""
    k4 = (k + 3) // 4 * 4
    us = (k + 1) // 2 * 2
    for n in range(1, NMAXW + 1):
        smem_cost = k4 * n * 4
        smem_grad = smem_cost + max(WT * (n + 1) + WT * us, WT * 8) * 4
        ys_end = k4 * n
        assert ys_end * 4 <= smem_cost
        hs_end = ys_end + WT * (n + 1)
        us_end = hs_end + WT * us
        assert us_end * 4 <= smem_grad <= 227 * 1024
        assert (hs_end * 4) % 8 == 0
    assert (k4 * 4) % 16 == 0   # row t of Ys starts 16-byte aligned for its float4 loads


# ---- the passes form (prost_wide.cu) -------------------------------------------

WIDE_CU = _src("prost_wide.cu")
KW = _const(DEVICE_H, r"constexpr int KMAX = (\d+);")
TOTF = _const(WIDE_CU, r"constexpr int TOTF = (\d+);")
assert "constexpr int NB4 = (KW / 4) * (KW / 4 + 1) / 2;" in WIDE_CU
assert "constexpr int GT = NB4 * 8;" in WIDE_CU
assert "constexpr int RS = KW + 4;" in WIDE_CU
assert "const int blk = t >> 3, g = t & 7;" in WIDE_CU
assert "for (int r = g; r < TILE_P; r += 8) {" in WIDE_CU
assert "part[(size_t)blockIdx.x * (k * (k + 1) / 2) + (i * k - i * (i - 1) / 2 + (j - i))] = s[p * 4 + q];" in WIDE_CU
MAX_CTAS = _const(WIDE_CU, r"constexpr int MAX_CTAS = (\d+);")
RCH = _const(WIDE_CU, r"constexpr int RCH = (\d+);")
GCH = _const(WIDE_CU, r"constexpr int GCH = (\d+);")
assert "const int c = u / nv, i = u - (u / nv) * nv;" in WIDE_CU
assert "constexpr int GPER = (KW * TILE_P + GT - 1) / GT;" in WIDE_CU
assert "v[q] = i < n ? __ldcg(src + i) : 0.f;" in WIDE_CU
assert "const int j = i / TILE_P, r = i - j * TILE_P;" in WIDE_CU and "tile[r * RS + j] = v[q];" in WIDE_CU
NB4 = (KW // 4) * (KW // 4 + 1) // 2
GT = NB4 * 8
RS = KW + 4


def _gram_block(blk):
    bi, rem = 0, blk
    while rem >= KW // 4 - bi:
        rem -= KW // 4 - bi
        bi += 1
    return bi, bi + rem


@pytest.mark.parametrize("k", range(1, KW + 1))
def test_wide_gram_writes_every_packed_entry_once(k):
    """Thread t of the Gram kernel sums the 4 x 4 block t / 8 over the rows
    r = t % 8 (mod 8); the lanes with t % 8 = 0 write the block's entries
    i <= j < k at the packed index of a k-wide upper triangle: every entry of
    that triangle exactly once, inside the NWG-float row."""
    nwg = KW * (KW + 1) // 2
    nm = k * (k + 1) // 2
    written = np.zeros(nm, np.int64)
    rows = np.zeros((NB4, TILE_P), np.int64)
    for t in range(GT):
        blk, g = t >> 3, t & 7
        bi, bj = _gram_block(blk)
        assert 0 <= bi <= bj < KW // 4
        i0, j0 = 4 * bi, 4 * bj
        # the 16-byte loads of a staged row stay inside it and aligned
        assert (i0 * 4) % 16 == 0 and (j0 * 4) % 16 == 0 and j0 + 4 <= RS
        if j0 >= k:
            continue
        rows[blk, g::8] += 1
        if g != 0:
            continue
        for p in range(4):
            for q in range(4):
                i, j = i0 + p, j0 + q
                if i <= j < k:
                    idx = i * k - i * (i - 1) // 2 + (j - i)
                    assert 0 <= idx < nm <= nwg
                    written[idx] += 1
    assert np.all(written == 1)
    used = sorted({_gram_block(t >> 3) for t in range(GT) if 4 * _gram_block(t >> 3)[1] < k})
    for blk in range(NB4):
        if _gram_block(blk) in used:
            assert np.all(rows[blk] == 1)  # each working block sums every row once
    assert TOTF >= nwg + 1


def test_wide_staged_tile_fits_and_rows_are_16_byte_aligned():
    # tile[r * RS + j] for r < TILE_P, j < k <= KW; each row starts on 16 bytes
    assert (RS * 4) % 16 == 0
    assert (TILE_P - 1) * RS + KW - 1 < TILE_P * RS
    # an 8-lane phase of 16-byte loads (one block, rows g + 8 it) touches 8
    # distinct 4-bank groups: bank of float (r * RS + i0) = (4 r + i0) mod 32
    for i0 in range(0, KW, 4):
        banks = {((g * RS + i0) % 32) // 4 for g in range(8)}
        assert len(banks) == 8


@pytest.mark.parametrize("ch,nv", [(RCH, KW + 3), (RCH, 1), (GCH, KW * (KW + 1) // 2), (GCH, 1)])
def test_wide_chunked_sum_reads_every_row_once(ch, nv):
    """chunked_sum: unit u = (chunk u / nv, value u % nv) loads rows
    chunk * CH + q < nrows of its value; every (row, value) exactly once,
    inside the nrows * nv partial floats, and the chunk sums fit the scratch
    sized for MAX_CTAS rows."""
    for nrows in (1, 2, 15, 16, 17, 39, 40, 41, 152, 303, 304, MAX_CTAS):
        nch = (nrows + ch - 1) // ch
        seen = np.zeros((nrows, nv), np.int64)
        for u in range(nv * nch):
            c, i = u // nv, u % nv
            assert c * nv + i < nv * ((MAX_CTAS + ch - 1) // ch)
            for q in range(ch):
                b = c * ch + q
                if b < nrows:
                    assert b * nv + i < nrows * nv
                    seen[b, i] += 1
        assert np.all(seen == 1)


@pytest.mark.parametrize("k", [1, 4, 5, 17, 31, 32])
def test_wide_gram_tile_copy_covers_the_block(k):
    """The Gram kernel's copy of one tile block: thread t's load q is entry
    i = t + GT q < k TILE_P of the block (column i / TILE_P, row i % TILE_P),
    stored transposed at r * RS + j: every entry once, inside the tile."""
    gper = (KW * TILE_P + GT - 1) // GT
    seen = np.zeros((KW, TILE_P), np.int64)
    n = k * TILE_P
    for t in range(GT):
        for q in range(gper):
            i = t + GT * q
            if i < n:
                j, r = i // TILE_P, i % TILE_P
                assert r * RS + j < TILE_P * RS
                seen[j, r] += 1
    assert np.all(seen[:k] == 1) and np.all(seen[k:] == 0)


# ---- the window pass's register-tiled dY product (prost_window.cu) ----------------

assert "constexpr int US = (K + 1) / 2 * 2, JP = US / 2;" in WINDOW_CU
assert "const int TQ = (n + 3) / 4, NB = JP * TQ, G = WT / NB;" in WINDOW_CU
assert "const int jp = bb / TQ, tq = bb - (bb / TQ) * TQ;" in WINDOW_CU
assert "red8[(g * NB + bb) * 8 + q] = dyacc[q];" in WINDOW_CU
assert "std::max((size_t)WT * (n + 1) + (size_t)WT * ((k + 1) / 2 * 2), (size_t)WT * 8)" in WINDOW_CU


@pytest.mark.parametrize("k", range(1, KMAXW + 1))
def test_window_dy_tiles_cover_every_entry_inside_the_scratch(k):
    """Thread bb + NB g of the gradient pass sums the 2 x 4 dY block bb
    (columns 2 jp, 2 jp + 1, frames 4 tq .. 4 tq + 3) over the rows r = g
    (mod G); every (column < k, frame < n) entry is written once, the pair
    loads stay inside the row tile, and the row groups' blocks (G x NB x 8
    floats) fit the eta and row tiles as the host sizes them."""
    us = (k + 1) // 2 * 2
    jp_n = us // 2
    for n in range(1, NMAXW + 1):
        tq_n = (n + 3) // 4
        nb = jp_n * tq_n
        g_n = WT // nb
        assert g_n >= 1
        grad_floats = max(WT * (n + 1) + WT * us, WT * 8)
        assert ((g_n - 1) * nb + nb - 1) * 8 + 7 < grad_floats
        seen = np.zeros((k, n), np.int64)
        for bb in range(nb):
            jp, tq = bb // tq_n, bb % tq_n
            assert 2 * jp + 1 < us
            for q in range(8):
                j, t = 2 * jp + q // 4, 4 * tq + (q & 3)
                if j < k and t < n:
                    seen[j, t] += 1
        assert np.all(seen == 1)


# ---- the resident form (k <= KREG): pixel units, item slots, shared memory ----

RES_UNIT = _const(DEVICE_H, r"constexpr int RES_UNIT = (\d+);")
assert "return (P + RES_UNIT - 1) / RES_UNIT;" in DEVICE_H
assert "return (int)((res_units(P) + G - 1) / G) * (RES_UNIT / 2);" in DEVICE_H
assert "const int64_t lo = nu * b / G, hi = nu * (b + 1) / G;" in FRAME_CUH
assert "ng = nitems > ns ? nitems - ns : 0;" in FRAME_CUH
assert "if (g > res_units(dp.P) + 1) g = res_units(dp.P) + 1;" in API_CU
# CTAs [0, G - 1) own the pixels; the end CTA G - 1 owns none
assert "const ResPart rpart(prm, G - 1, b, a.res_ns);" in FRAME_CUH
assert "const int npm = res_npair_max(P, grid - 1);" in FRAME_CUH
# the partial buffers: two per launch, and in the resident form RES_NREP copies
# of each pass's partial values (CTA b writes every copy, reads copy b % RES_NREP)
RES_NREP = _const(DEVICE_H, r"constexpr int RES_NREP = (\d+);")
assert "(size_t)2 * RES_NREP * col_stride(h->grid_res) * partial_row(prm->k));" in API_CU
assert "float *const bbase = a.partials + (size_t)buf * NREP * F::NVR * cs;" in FRAME_CUH
assert "const float *cols = bbase + (size_t)(b % NREP) * F::NVR * cs;" in FRAME_CUH


def res_units(P):
    return (P + RES_UNIT - 1) // RES_UNIT


def res_npair_max(P, G):
    return -(-res_units(P) // G) * (RES_UNIT // 2)


def al16(b):
    return (b + 15) // 16 * 16


def res_part(P, C, G, b, ns):
    nu = res_units(P)
    lo, hi = nu * b // G, nu * (b + 1) // G
    pa = lo * RES_UNIT
    pb = min(hi * RES_UNIT, P)
    npair = (max(pb - pa, 0) + 1) // 2
    nitems = C * npair
    return pa, npair, nitems, max(nitems - ns, 0)


RES_CPL = _const(DEVICE_H, r"constexpr int RES_CPL = (\d+);")
RES_VPW = _const(DEVICE_H, r"constexpr int RES_VPW = (\d+);")
assert "constexpr int RES_MAX_GRID = 128 * RES_CPL;" in DEVICE_H
assert "if (g > RES_MAX_GRID) g = RES_MAX_GRID;" in API_CU


def res_plan(P, C, k, usz, fsz, cap):
    """Grid, row slots and dynamic shared memory as FrameOps::res_plan_t sizes them."""
    G = min(SMS, res_units(P) + 1, RED_SCR // partial_row(k) * RED_ROWS, 128 * RES_CPL)
    if G < 2:
        return None
    npm = res_npair_max(P, G - 1)
    fixed = al16(C * npm * 2 * fsz) + al16(npm * 2)
    if cap <= fixed:
        return None
    ns = min(C * npm, (cap - fixed) // (k * 2 * usz))
    smem = al16(k * ns * 2 * usz) + fixed
    assert smem <= cap
    return G, ns, npm, smem


RES_CASES = [(P, C) for P in (1, 2, 63, 64, 65, 1073, 2000, 19200, 76800, 307200, 921600, 2073600)
             for C in (1, 3)]


@pytest.mark.parametrize("P,C", RES_CASES)
@pytest.mark.parametrize("k,usz,fsz", [(10, 4, 1), (10, 4, 4), (10, 2, 1), (5, 4, 4), (1, 4, 1)])
@pytest.mark.parametrize("cap", [219648, 40000])
def test_resident_plan_covers_every_entry_once_inside_its_buffers(P, C, k, usz, fsz, cap):
    plan = res_plan(P, C, k, usz, fsz, cap)
    if plan is None:
        return
    G, ns, npm, smem = plan
    npt = npt_of(P)
    Pp = npt * TILE_P
    seen = np.zeros((C, P), dtype=np.int32)
    nt = threads(k, usz == 2)
    for b in range(G):
        pa, npair, nitems, ng = res_part(P, C, G - 1, b, ns)
        assert npair <= npm and nitems <= C * npm
        if b == G - 1:
            assert nitems == 0  # the end CTA streams no rows
        if nitems == 0:
            continue
        assert pa % 2 == 0
        it = np.arange(nitems)
        c, q = it // npair, it % npair
        p = pa + 2 * q
        nvalid = np.minimum(2, P - p)
        assert (nvalid >= 1).all()
        np.add.at(seen, (c, p), 1)
        two = nvalid == 2
        np.add.at(seen, (c[two], p[two] + 1), 1)
        # global row pairs: 8 (float32) or 4 (bfloat16) bytes at an even entry of a tile column
        pt = p // TILE_P
        r = p - pt * TILE_P
        base = (c * npt + pt) * k * TILE_P + r
        assert (r % 2 == 0).all() and (r + 1 < TILE_P).all()
        assert (base + (k - 1) * TILE_P + 1 < C * npt * k * TILE_P).all()
        # frame pairs (16-byte aligned planes, pitch P or Pp) and label pairs
        assert (p + 1 < Pp).all() and (p[two] + 1 < P).all()
        # shared memory: slots of items [ng, nitems), frame entries of every item,
        # labels of every pair; each region inside the dynamic allocation
        s = it[it >= ng] - ng
        assert (s < ns).all()
        assert al16(k * ns * 2 * usz) + al16(C * npm * 2 * fsz) + npm * 2 <= smem
        assert it.max() < C * npm and q.max() < npm
        # each thread's incremental (c, q) walk lands on item c npair + q
        for t in range(min(nt, nitems)):
            cc, qq = 0, t
            while qq >= npair and cc < C:
                qq -= npair
                cc += 1
            for i in range(t, nitems, nt):
                assert i == cc * npair + qq
                qq += nt
                while qq >= npair and cc < C:
                    qq -= npair
                    cc += 1
    assert (seen == 1).all()
    # the warps' cross-CTA sums: every value has a warp, every CTA's entry a
    # lane's chunk, and each 16-byte chunk ends inside the value's row
    nvals = partial_row(k)
    assert nvals <= RES_VPW * (threads(k, usz == 2) // 32)
    nch = (G + 3) // 4
    assert nch <= 32 * RES_CPL and 4 * nch <= (G + 3) // 4 * 4
    # partial values of every pass: copy r of value c of CTA b inside the buffers
    cs = (G + 3) // 4 * 4
    nv = partial_row(k)
    floats = 2 * RES_NREP * cs * nv
    for buf in (0, 1):
        base = buf * RES_NREP * nv * cs
        top = max(base + r * nv * cs + c * cs + b for r in (0, RES_NREP - 1) for c in (0, nv - 1)
                  for b in (0, G - 1))
        assert top < floats


# ---- the resident form's multi-frame launches --------------------------------

assert "const int64_t np = prm.P - rp.pa < 2 * (int64_t)rp.npair ? prm.P - rp.pa : 2 * (int64_t)rp.npair;" in FRAME_CUH
assert "const int nl = (int)((bytes + 127) / 128);" in FRAME_CUH
assert "if (left >= 1 && run > left) run = (int32_t)left;" in API_CU


@pytest.mark.parametrize("P,C", [(1, 1), (15, 3), (1073, 3), (19200, 1), (307200, 3)])
@pytest.mark.parametrize("fsz", [1, 4])
def test_next_frame_prefetch_stays_in_the_next_frame(P, C, fsz):
    """res_prefetch_frame: one 128-byte line per (channel, line of the CTA's
    pixels), each address inside the CTA's range of that plane of the next
    frame, for planes P (direct) or Pp (staged) entries apart."""
    G = min(SMS, res_units(P) + 1)
    for pitch in {P, npt_of(P) * TILE_P}:
        for b in range(G):
            pa, npair, _, _ = res_part(P, C, G - 1, b, 0)
            n = min(P - pa, 2 * npair)
            if n <= 0:
                continue
            nl = (n * fsz + 127) // 128
            for c in range(C):
                lines = pa * fsz + c * pitch * fsz + 128 * np.arange(nl)
                assert lines.min() >= (c * pitch + pa) * fsz
                assert lines.max() < (c * pitch + pa + n) * fsz


@pytest.mark.parametrize("since", [0, 1, 1000, 1023])
@pytest.mark.parametrize("n", [1, 16, 25, 2049])
def test_multi_frame_calls_split_at_the_rebase(since, n):
    """prost_step_many / prost_step_many_async: runs of frames in one launch
    each, none crossing the every-1,024-frames rebase; together they cover the
    call's frames in order."""
    rebase = _const(DEVICE_H, r"constexpr uint32_t REBASE_EVERY = (\d+);")
    s, i0, runs = since, 0, []
    while i0 < n:
        run = n - i0
        left = rebase - s
        if left >= 1 and run > left:
            run = left
        runs.append((i0, run))
        s += run
        if s >= rebase:
            s = 0
        i0 += run
    assert sum(r for _, r in runs) == n and all(r >= 1 for _, r in runs)
    # every run ends at or before the next rebase
    s = since
    for _, run in runs:
        assert s + run <= rebase
        s = (s + run) % rebase


def test_next_frame_coefficients_repeat_the_end_of_frame_fold():
    """The resident form's CTAs form the next frame's stored-row coefficients
    T_old y themselves, with the same FP64 operations in the same order as
    end_frame, so that a multi-frame launch reproduces one launch per frame
    bit for bit (the GPU test of that is tests/test_gpu_many.py)."""
    handover = "for (int q = tid; q < K; ++q) ty = dfma(rs.Told[tid * K + q], sk.y[q], ty);"
    fold = "for (int q = t; q < K; ++q) ty = dfma(rs.Told[t * K + q], sk.y[q], ty);"
    assert handover in FRAME_CUH and fold in FRAME_CUH
    assert "sk.yf[tid] = (float)ty;" in FRAME_CUH and "ks->yf[t] = (float)rs.ty[t];" in FRAME_CUH
