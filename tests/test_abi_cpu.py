"""The C-ABI library builds, loads and exports every declared symbol (CPU only;
no kernel is launched)."""
import ctypes
import os
import re

import pytest

import paper_0909_2000_gb300 as ap

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    text = ""
    inc = os.path.join(ROOT, "include")
    for f in sorted(os.listdir(inc)):
        if f.endswith(".h"):
            text += open(os.path.join(inc, f)).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(ap_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for s in ["ap_alignment_plot", "ap_alignment_dots", "ap_plot_shape", "ap_plot_plan",
              "ap_dots_workspace_size", "ap_plot_checksum", "ap_last_error"]:
        assert s in syms


def test_library_exports_every_declared_symbol():
    lib = ap.load()
    raw = ctypes.CDLL(ap.library_path())
    missing = [s for s in declared_symbols() if not hasattr(raw, s)]
    assert missing == []
    assert "sm_103a" in ap.version()
    assert lib is ap.load()


def test_host_side_validation_without_gpu():
    assert ap.plot_shape(512, 512, 16) == (496, 496)
    assert ap.plot_shape(5, 9, 5) == (0, 4)
    with pytest.raises(ap.ApError) as e:
        ap.plot_shape(10, 10, 0)
    assert e.value.status == ap.AP_E_INVAL
    with pytest.raises(ap.ApError) as e:
        ap.plot_plan(100, 100, 10, (9, 1, 0))      # reduced form {9,1,0}: not built
    assert e.value.status == ap.AP_E_UNSUPPORTED
    with pytest.raises(ap.ApError) as e:
        ap.plot_plan(100, 100, 10, (10, 3, 0))     # reduced form {10,3,0}: not built
    assert e.value.status == ap.AP_E_UNSUPPORTED
    with pytest.raises(ap.ApError) as e:
        ap.plot_plan(1000, 1000, 193, (5, 1, 0))   # nu = 5: w <= 192
    assert e.value.status == ap.AP_E_UNSUPPORTED
    with pytest.raises(ap.ApError) as e:
        ap.plot_plan(1000, 1000, 257, (3, 1, 0))   # beyond the compiled windows
    assert e.value.status == ap.AP_E_UNSUPPORTED
    with pytest.raises(ap.ApError) as e:
        ap.plot_plan(100, 100, 10, (1, 1, 0))     # not normalised
    assert e.value.status == ap.AP_E_INVAL
    with pytest.raises(ap.ApError) as e:
        ap.plot_plan(100, 100, 10, (1, 0, -1))
    assert e.value.status == ap.AP_E_INVAL
    with pytest.raises(ap.ApError) as e:
        ap.plot_plan(100000, 100000, 600)
    assert e.value.status == ap.AP_E_UNSUPPORTED
    for w, sc in ((513, ap.LCS), (257, ap.SCORE)):    # one past the largest windows built
        with pytest.raises(ap.ApError) as e:
            ap.plot_plan(2000, 2000, w, sc)
        assert e.value.status == ap.AP_E_UNSUPPORTED
    with pytest.raises(ap.ApError):
        ap.set_chunk(-1)


@pytest.mark.parametrize("w,scores", [(1, ap.LCS), (16, ap.LCS), (100, ap.LCS), (120, ap.LCS),
                                      (121, ap.LCS), (128, ap.LCS), (129, ap.LCS), (240, ap.LCS),
                                      (241, ap.LCS), (254, ap.LCS),
                                      (255, ap.LCS), (256, ap.LCS), (257, ap.LCS), (300, ap.LCS), (384, ap.LCS),
                                      (480, ap.LCS), (481, ap.LCS), (512, ap.LCS), (1, ap.SCORE),
                                      (64, ap.SCORE), (65, ap.SCORE), (120, ap.SCORE),
                                      (121, ap.SCORE), (254, ap.SCORE), (256, ap.SCORE)])
def test_every_supported_window_has_a_variant(w, scores):
    pl = ap.plot_plan(w + 1000, w + 777, w, scores)
    rows = 2 * w if scores == ap.SCORE else w
    assert pl["comb_rows"] == rows
    assert pl["rows_per_lane"] * pl["lanes_per_strip"] >= rows
    assert pl["logical_cells"] == 1000 * 777 * w
    # key width: 7-bit up to w = 120, then full 8-bit lanes up to 240 (LCS only;
    # up to 254 on request), 16-bit lanes otherwise (10-bit lanes only on
    # request)
    lcs = scores == ap.LCS
    want = 8 if (w <= 120 or (w <= 240 and lcs)) else 16
    assert pl["lane_bits"] == want
    assert pl["strips_per_reg"] == {8: 4, 10: 3, 16: 2}[want]
    assert pl["physical_cells"] >= pl["logical_cells"] * (4 if scores == ap.SCORE else 1)


@pytest.mark.parametrize("nu,mu", [(3, 1), (3, 2), (4, 1), (4, 2), (4, 3), (2, 0), (7, 0), (6, 3), (6, 2),
                                   (8, 6), (12, 3), (5, 1), (5, 4), (6, 1), (6, 5), (7, 2), (7, 6),
                                   (8, 3), (8, 7), (10, 4), (16, 2)])
@pytest.mark.parametrize("w", [1, 7, 32, 33, 64, 128, 200, 256])
def test_blown_up_score_schemes_have_variants(nu, mu, w):
    """Schemes reduce by g = gcd(match, mismatch); the reduced blow-up is
    combed, so the comb height is (match / g) * w."""
    import math
    g = math.gcd(nu, mu)
    rn = nu // g
    # largest windows built: LCS 512, {2,1,0} 256, nu = 3, 4: 256, then
    # 8 threads of at most 128 rows: 192 (nu = 5), 160 (6), 128 (7, 8)
    if w > {1: 512, 2: 256, 3: 256, 4: 256, 5: 192, 6: 160, 7: 128, 8: 128}[rn]:
        with pytest.raises(ap.ApError):
            ap.plot_plan(w + 500, w + 300, w, (nu, mu, 0))
        return
    pl = ap.plot_plan(w + 500, w + 300, w, (nu, mu, 0))
    assert pl["comb_rows"] == rn * w
    assert pl["rows_per_lane"] * pl["lanes_per_strip"] >= rn * w
    assert pl["physical_cells"] >= pl["logical_cells"] * rn * rn


def test_scores_whose_plot_exceeds_16_bits_are_refused():
    import ctypes
    sc = ap._scores((1000, 0, 0))          # 1000 x LCS: values up to 100,000
    with pytest.raises(ap.ApError) as e:
        ap._check(ap.load().ap_alignment_plot(None, 1000, None, 1000, 100, ctypes.byref(sc), None, 2, 900, None))
    assert e.value.status == ap.AP_E_INVAL


def test_plan_of_the_100k_plot():
    pl = ap.plot_plan(100_000, 100_000, 100)
    assert pl["lane_bits"] == 8 and pl["strips_per_reg"] == 4 and pl["lanes_per_strip"] == 1
    # warm-up and padding overhead stay small
    assert pl["physical_cells"] < 1.06 * pl["logical_cells"]


def test_chunk_count_minimises_rounds_times_tile_length():
    """tile_plan's choice (host-only planning assumes 152 SMs x 8 warps): the
    chunk count minimises ceil(tiles / S) * (chunk + w - 1 + 8) over every
    count that gives a distinct 32-aligned chunk."""
    S = 152 * 8
    for m, n, w in ((100_000, 100_000, 100), (20_000, 20_000, 100), (512, 512, 16),
                    (100_000, 100_000, 16), (3000, 90_000, 64)):
        pl = ap.plot_plan(m, n, w)
        rows, cols = ap.plot_shape(m, n, w)
        nsg = -(-rows // (pl["strips_per_reg"] * 32 // pl["lanes_per_strip"]))

        def cost(ch):
            nch = -(-cols // ch)
            return -(-(nsg * nch) // S) * (ch + w - 1 + 8)
        chunks = {-(-(-(-cols // k)) // 32) * 32 for k in range(1, cols // 32 + 2)}
        best = min(cost(ch) for ch in chunks)
        assert pl["chunk"] % 32 == 0
        assert cost(pl["chunk"]) <= best * (1 + 1e-9), (m, n, w, pl["chunk"])


def test_band_rows_override_sets_the_banded_workspaces():
    """ap_set_band_rows (host only): the dots workspace holds one band, so its
    size follows the forced band height, rounded up to whole strip groups."""
    base = ap._scores(ap.LCS)
    import ctypes
    lib = ap.load()

    def ws(m, n, w):
        b = ctypes.c_int64()
        ap._check(lib.ap_dots_workspace_size(m, n, w, ctypes.byref(base), ctypes.byref(b)))
        return b.value
    auto = ws(5000, 5000, 40)
    try:
        ap.set_band_rows(100)           # 128-strip groups: one group per band
        small = ws(5000, 5000, 40)
        ap.set_band_rows(129)           # two groups
        two = ws(5000, 5000, 40)
    finally:
        ap.set_band_rows(0)
    assert small < two < auto == ws(5000, 5000, 40)
    with pytest.raises(ap.ApError) as e:
        ap.set_band_rows(-1)
    assert e.value.status == ap.AP_E_INVAL


def test_release_build_has_no_bounds_checks():
    with pytest.raises(ap.ApError) as e:
        ap.debug_bounds()
    assert e.value.status == ap.AP_E_UNSUPPORTED


@pytest.mark.parametrize("bits,g,w", [(10, 4, 128), (10, 4, 200), (16, 4, 128), (8, 4, 200), (16, 8, 100)])
def test_lane_format_switch(bits, g, w):
    try:
        ap.set_lane_bits(bits)
        ap.set_lanes_per_strip(g)
        pl = ap.plot_plan(w + 500, w + 400, w)
    finally:
        ap.set_lane_bits(0)
        ap.set_lanes_per_strip(0)
    assert pl["lane_bits"] == bits and pl["lanes_per_strip"] == g
    assert pl["rows_per_lane"] * g >= w
    with pytest.raises(ap.ApError):
        ap.set_lane_bits(12)


@pytest.mark.parametrize("w", [1, 5, 10, 15, 16, 40, 100, 128, 200, 256, 300, 480])
@pytest.mark.parametrize("bits", [0, 8, 10, 16])
@pytest.mark.parametrize("g", [0, 1, 2, 4, 8])
def test_requested_layouts_keep_padding_within_the_masked_rows(w, bits, g):
    """Any lane-format and threads-per-strip request yields a plan whose
    threads each hold their share of the window with at most the masked
    padding rows (else the automatic choice): rows_per_lane * groups covers
    w, and no thread's share falls more than 8 rows short of its rows."""
    try:
        ap.set_lane_bits(bits)
        ap.set_lanes_per_strip(g)
        pl = ap.plot_plan(w + 700, w + 600, w)
    finally:
        ap.set_lane_bits(0)
        ap.set_lanes_per_strip(0)
    G, R = pl["lanes_per_strip"], pl["rows_per_lane"]
    assert R * G >= w and R - w // G <= 8, pl


@pytest.mark.parametrize("bits", [0, 8, 10, 16])
@pytest.mark.parametrize("g", [0, 1, 2, 4, 8])
def test_every_lcs_layout_has_match_tables(bits, g):
    """Every LCS plan, automatic or requested, has match tables for warps of
    at most four letters: on one thread (7-bit keys), or shared by the G
    threads of a strip group with g w / G rounded down (2) or up (3) to whole
    table loads (4, 2, 1 rows for 8-, 16-, 10-bit lanes) as the first row of
    thread g; each thread's share then holds at most its R rows and at most
    8 (the masked padding rows) fewer."""
    try:
        ap.set_lane_bits(bits)
        ap.set_lanes_per_strip(g)
        plans = {w: ap.plot_plan(w + 700, w + 600, w) for w in range(1, 513)}
    finally:
        ap.set_lane_bits(0)
        ap.set_lanes_per_strip(0)
    for w, pl in plans.items():
        G, R, t = pl["lanes_per_strip"], pl["rows_per_lane"], pl["tables"]
        if G == 1:
            assert t == 1 and pl["lane_bits"] == 8, (w, pl)
            continue
        assert t in (2, 3), (w, pl)
        rpl = {8: 4, 16: 2, 10: 1}[pl["lane_bits"]]
        ub = [(-(-(k * w) // G) + rpl - 1) // rpl * rpl if t == 3 else (k * w // G) // rpl * rpl
              for k in range(G)] + [w]
        shares = [ub[k + 1] - ub[k] for k in range(G)]
        assert all(R - 8 <= s <= R for s in shares), (w, pl, shares)


def test_issue_probe_validates_before_touching_a_device():
    for kind, iters in ((3, 10), (-1, 10), (0, 0)):
        with pytest.raises(ap.ApError) as e:
            ap.int_issue_probe(kind, iters)
        assert e.value.status == ap.AP_E_INVAL


@pytest.mark.parametrize("bits", [0, 8, 10, 16])
@pytest.mark.parametrize("g", [0, 1, 2, 4, 8])
def test_every_plan_fits_the_shared_memory_of_a_block(bits, g):
    """Every plan, LCS or score, automatic or requested, asks a block for at
    most 227 KB of shared memory (the sm_103a limit), so every launch can
    run; the 100k bench plot fits two blocks per SM."""
    plans = []
    try:
        ap.set_lane_bits(bits)
        ap.set_lanes_per_strip(g)
        for w in range(1, 513):
            for sc in (ap.LCS, ap.SCORE, (3, 1, 0), (5, 2, 0), (8, 7, 0)):
                try:
                    plans.append((w, sc, ap.plot_plan(w + 700, w + 600, w, sc)))
                except ap.ApError:
                    pass
    finally:
        ap.set_lane_bits(0)
        ap.set_lanes_per_strip(0)
    assert plans
    for w, sc, pl in plans:
        assert 0 < pl["smem_per_block"] <= 227 * 1024, (w, sc, pl)
    assert 2 * ap.plot_plan(100_000, 100_000, 100)["smem_per_block"] <= 228 * 1024
