"""The blends' lane geometry, checked on the host without a GPU.

The forward's staging test clears band bit w G + g when no pixel of the
rectangle GroupRect(w, g) can meet a primitive, and lane group g of warp w
then skips the entry; the forward writes one contributor-mask row per lane
group and the backward's groups walk their own rows.  That is only right if
the lanes that LaneGroups puts in group g of warp w are exactly the pixels of
GroupRect(w, g) under WarpGrid's pixel layout, if each group has one leader
(its lowest lane, which writes the group's mask word), and if the OR
reduction's lane partners stay inside the group.

A small host program built with nvcc from the kernels' own headers
(WarpGrid::pixel, LaneGroups and GroupRect are host-callable) checks this for
every (tile edge, pixels per thread) schedule that is built.  It needs nvcc
but no GPU."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2501_16312_gb300", "csrc")

PROBE = r"""
#include <cstdio>
#include "lp_blend.cuh"
using namespace lp;

template <int TILE, int PIX> int check() {
    using WG = WarpGrid<TILE, PIX>;
    using LG = LaneGroups<TILE, PIX>;
    using R = GroupRect<TILE, PIX>;
    int bad = 0;
    if (WG::NW * LG::G > 64) ++bad;
    for (int w = 0; w < WG::NW; ++w)
        for (int g = 0; g < LG::G; ++g) {
            static int hit[32][32];
            for (int y = 0; y < 32; ++y) for (int x = 0; x < 32; ++x) hit[y][x] = 0;
            int leaders = 0, lowest = -1;
            for (int lane = 0; lane < 32; ++lane) {
                if (LG::group(lane) != g) continue;
                if (lowest < 0) lowest = lane;
                if (LG::leader(lane)) { ++leaders; if (lane != lowest) ++bad; }
                int ly, lx0;
                WG::pixel(w * 32 + lane, ly, lx0);
                for (int i = 0; i < PIX; ++i) hit[ly][lx0 + i] += 1;
                for (int b = 0; b < 5; ++b)   // partners of the OR reduction
                    if (!((LG::kGroupBits >> b) & 1u) && LG::group(lane ^ (1 << b)) != g) ++bad;
            }
            if (leaders != 1) ++bad;
            for (int y = 0; y < TILE; ++y)
                for (int x = 0; x < TILE; ++x) {
                    const bool in = x >= R::x0(w, g) && x < R::x0(w, g) + R::GW &&
                                    y >= R::y0(w, g) && y < R::y0(w, g) + R::GH;
                    if (hit[y][x] != (in ? 1 : 0)) ++bad;
                }
        }
    std::printf("%d %d %d %d %d\n", TILE, PIX, WG::NW, LG::G, bad);
    return bad;
}

int main() {
    int bad = 0;
    if constexpr (tile_pix_ok(8, 1)) bad += check<8, 1>();
    if constexpr (tile_pix_ok(8, 2)) bad += check<8, 2>();
    if constexpr (tile_pix_ok(16, 1)) bad += check<16, 1>();
    if constexpr (tile_pix_ok(16, 2)) bad += check<16, 2>();
    if constexpr (tile_pix_ok(16, 4)) bad += check<16, 4>();
    if constexpr (tile_pix_ok(32, 2)) bad += check<32, 2>();
    if constexpr (tile_pix_ok(32, 4)) bad += check<32, 4>();
    return bad != 0;
}
"""


def _nvcc():
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    return None


def test_lane_groups_cover_their_rectangles(tmp_path):
    nvcc = _nvcc()
    if nvcc is None:
        pytest.skip("nvcc not found")
    src = tmp_path / "lane_probe.cu"
    exe = tmp_path / "lane_probe"
    src.write_text(PROBE)
    subprocess.check_call([nvcc, "-std=c++17", "--expt-relaxed-constexpr", "-I", os.path.join(ROOT, "include"),
                           "-I", CSRC, str(src), "-o", str(exe)])
    out = subprocess.run([str(exe)], capture_output=True, text=True)
    rows = [list(map(int, line.split())) for line in out.stdout.splitlines()]
    assert rows, out.stdout + out.stderr
    seen = {(t, p) for t, p, _, _, _ in rows}
    assert {(8, 1), (16, 2), (16, 4), (32, 4)} <= seen, seen
    for tile, pix, nw, g, bad in rows:
        assert g == 4 and nw * g <= 64, (tile, pix, nw, g)
        assert bad == 0, (tile, pix, bad)
    assert out.returncode == 0
