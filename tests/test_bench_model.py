"""The benchmark's algorithmic work model (the numerator of its roofline) against
counts derived here from first principles.

Double-float primitives (two_sum, fast_two_sum, df_add, df_mul) are counted from their
definitions as FP32 operations; a length-n power-of-two transform built from radix-8
passes and one radix-4 or radix-2 pass is counted butterfly by butterfly, with an
r-point radix-2 DFT taking r log2(r) complex additions and the k = 0 twiddles of each
pass free.
"""
import math
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402

TWO_SUM = 6          # s, bb, and four operations for the error term
FAST_TWO_SUM = 3
DF_ADD = TWO_SUM + 2 + FAST_TWO_SUM          # two-sum of the highs, two adds of the lows, renormalise
DF_MUL = 1 + 3 + FAST_TWO_SUM                # product, three fused multiply-adds, renormalise
CADD = 2 * DF_ADD
CMUL = 4 * DF_MUL + 2 * DF_ADD
MUL_W8 = 2 * DF_ADD + 2 * DF_MUL             # (re +- im) / sqrt(2)


DF_HALF = 2                                  # both words times 0.5 (exact)


def dft_ops(r):
    if r == 3:
        # t1 = v1 + v2; t2 = v0 - t1/2; t3 = -+i (sqrt(3)/2)(v1 - v2); y0 = v0 + t1, y1,2 = t2 +- t3
        return 5 * CADD + 2 * DF_ADD + 2 * DF_HALF + 2 * DF_MUL
    adds = r * int(math.log2(r))
    extra = 2 * MUL_W8 if r == 8 else 0      # w8 and w8^3 (w8^2 = -i costs nothing)
    return adds * CADD + extra


def transform_ops_per_point(n):
    """Walk the passes of a length-n transform point by point (a radix-3 pass first
    when 3 divides n)."""
    three = n % 3 == 0
    l = int(round(math.log2(n // 3 if three else n)))
    radices = ([3] if three else []) + [8] * (l // 3) + ([2 ** (l % 3)] if l % 3 else [])
    total, ns = 0, 1
    for r in radices:
        butterflies = n // r
        nontrivial = butterflies - butterflies // ns          # k = 0 butterflies have unit twiddles
        total += nontrivial * (r - 1) * CMUL + butterflies * dft_ops(r)
        ns *= r
    return total / n


def test_primitive_counts_match_the_model():
    assert DF_ADD == 11 and DF_MUL == 7 and CMUL == bench.DF_CMUL == 50
    for r in (2, 3, 4, 8):
        assert bench.DF_DFT[r] == dft_ops(r), r


@pytest.mark.parametrize("n", [16, 32, 48, 64, 96, 128, 192, 256, 384, 512, 768, 1024])
def test_transform_ops_per_point(n):
    assert bench.df_transform_ops(n) == pytest.approx(transform_ops_per_point(n), rel=1e-12)


def test_z_pass_work_of_the_charged_sphere_mesh():
    """Forward and inverse z transforms plus the Green's scaling (two df_mul per point)
    on the half spectrum of the 128^3 mesh: 515.2 M FP32 operations per launch; its
    algorithmic bytes: the double-float half spectrum (16 B per point) read and written
    and the double-float Green's table (8 B per point) read, 34.1 MB + 5.3 MB."""

    class S:
        mesh = (128, 128, 128)
        n = 0

    pts = 128 * 128 * 65
    ops = bench.alu_work(S)
    assert ops == pytest.approx(pts * (2 * transform_ops_per_point(128) + 2 * DF_MUL), rel=1e-12)
    assert ops == pytest.approx(515.2e6, rel=1e-3)
    bound, work, unit = bench.stage_work("scale64", S, 0, True)
    assert bound == "hbm" and unit == "GB/s" and work == pts * (2 * 16 + 8)


def test_pme_bytes_of_the_lattice():
    """6 G w R + N (32 + 8 R) for the 256^3 FP32 mesh and 141,088 beads, one field."""

    class S:
        mesh = (256, 256, 256)
        n = 141_088

    assert bench.pme_bytes(S) == 6 * 256 ** 3 * 4 + 141_088 * 40


@pytest.mark.parametrize("n,ok", [(16, True), (24, True), (40, False), (48, True), (96, True), (192, True), (256, True),
                                  (768, True), (1024, True), (1536, False), (12, False), (8, False), (100, False)])
def test_double_float_mesh_rule(n, ok):
    """2^k or 3 2^k with a power-of-two part of at least 8, 16 to 1024 points."""
    assert bench.df_mesh_size(n) == ok
