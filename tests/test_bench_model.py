"""The bench's per-kernel roofline model (host logic, no GPU): every kernel
name that `csl_time_kernels` reports for a 2D or 3D plan gets its own model
entry, with the algorithmic bytes per point of that kernel, and the bound
follows from comparing bytes and flops against the peaks."""
import os
import sys

import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402

M = 1023 * 1023
NAMES_2D = ["k_stencil", "k_row<LOAD_LANCZOS,STORE_T>", "k_strided<mid>", "k_row<LOAD_T,STORE_Z>", "k_update"]


@pytest.mark.parametrize("prec,sT", [("fp32", 8), ("fp64", 16)])
def test_bytes_per_point(prec, sT):
    per = {nm: bench.kernel_model(nm, M, 2, prec, 1024, ff=(prec == "fp32"))[0] / M for nm in NAMES_2D}
    # float-pair stencil: z, v_{j-1} in, u' out, 2 face pairs; FP64: + diagonal, 2 FP64 faces
    assert per["k_stencil"] == (sT + 16 + 16 + 16 if prec == "fp32" else sT + 16 + 16 + 8 + 16)
    assert per["k_row<LOAD_LANCZOS,STORE_T>"] == 16 + 16 + 16 + sT
    assert per["k_strided<mid>"] == 2 * sT + (8 if prec == "fp64" else 0)
    assert per["k_row<LOAD_T,STORE_Z>"] == 2 * sT
    assert per["k_update"] == sT + 80


def test_fp32_precond_form_bytes_and_fp64_work():
    # FP32 transforms (8-byte T, z), FP64 vectors: the stencil reads an FP32 z
    # and FP64 faces/diagonal; the Lanczos step and the update are FP64
    per = {nm: bench.kernel_model(nm, M, 2, "fp32_precond", 1024) for nm in NAMES_2D}
    assert per["k_stencil"][0] / M == 8 + 16 + 16 + 8 + 16 and per["k_stencil"][1] > 0
    assert per["k_row<LOAD_LANCZOS,STORE_T>"][0] / M == 16 + 16 + 16 + 8
    assert per["k_row<LOAD_LANCZOS,STORE_T>"][1] / M == 4
    assert per["k_update"][0] / M == 8 + 80 and per["k_update"][1] > 0
    assert per["k_strided<mid>"][0] / M == 16 and per["k_strided<mid>"][1] == 0


def test_fp32_forms_have_no_fp64_vector_work():
    for nm in NAMES_2D:
        _, f64, _ = bench.kernel_model(nm, M, 2, "fp32", 1024, ff=True)
        assert f64 == 0, nm


def test_bound_and_fraction():
    # 1 ms per kernel: every kernel is far from its roof, and frac = achieved / peak
    rows = bench.roofline_table([(nm, 1.0) for nm in NAMES_2D], M, 2, "fp32", 1023, 6800.0, 186, ff=True)
    by = {r["kernel"]: r for r in rows}
    assert by["k_update"]["bound"] == "hbm"
    assert by["k_update"]["achieved"] == pytest.approx(88 * M / 1e-3 / 1e9, rel=1e-3)
    for r in rows:  # the table rounds frac to 4 decimals
        assert r["frac"] == pytest.approx(r["achieved"] / r["peak"], abs=1e-4)
    assert abs(sum(x["share"] for x in rows) - 1.0) < 1e-3
