"""The roofline arithmetic used by the benchmark report, pinned to numbers
printed in the paper (Table 1, Sec. 4.3 after Eq. 9, Table 2, App. A.5)."""
import os

import pytest

from paper_2206_14286_gb300 import roofline as RF


def golden():
    out = {}
    path = os.path.join(os.path.dirname(__file__), "golden", "paper_numbers.txt")
    for line in open(path):
        line = line.split("#")[0].strip()
        if line:
            k, v = line.split()
            out[k] = float(v)
    return out


G = golden()


def test_cop_budget_d128():
    # Sec. 4.3: "4 ... for TPU V4, and 16 for GPU A100" at D = 128
    v4 = RF.cop_budget(128, G["tpuv4_gamma"], G["tpuv4_pi"])
    a100 = RF.cop_budget(128, G["a100_gamma"], G["a100_pi"])
    assert round(v4) == G["cop_budget_d128_tpuv4"]
    assert a100 == pytest.approx(G["cop_budget_d128_a100"], rel=1e-12)


def test_icop_table2():
    assert RF.i_cop(G["glove_D"], G["glove_C"]) == pytest.approx(G["glove_icop"], abs=0.05)
    assert RF.i_cop(G["sift_D"], G["sift_C"]) == pytest.approx(G["sift_icop"], abs=0.05)


def test_sift_cop_bound_binds_on_v4_not_v3():
    """Fig. 2 discussion / App. A.5: Sift (C = 6) is COP-bound on TPU V4 only."""
    icop = RF.i_cop(G["sift_D"], G["sift_C"])
    big_imem = 4701.0  # Table 2, profiler value
    v4 = RF.binding_roof(G["tpuv4_pi"], G["tpuv4_beta"] / 1e3, G["tpuv4_gamma"], big_imem, icop)
    v3 = RF.binding_roof(G["tpuv3_pi"], G["tpuv3_beta"] / 1e3, G["tpuv3_gamma"], big_imem, icop)
    assert v4 == "cop" and v3 == "tensor"
    # Glove (C = 4) stays under pi on both
    icop_g = RF.i_cop(G["glove_D"], G["glove_C"])
    assert RF.binding_roof(G["tpuv4_pi"], G["tpuv4_beta"] / 1e3, G["tpuv4_gamma"], 4758.0, icop_g) == "tensor"


def test_eq7_dense_scores_intensity():
    assert RF.i_mem_dense_scores(10000, 10 ** 6, 128) == pytest.approx(128 / 2)


def test_eq20_approaches_min_m_n():
    a = RF.i_mem_partial_reduce(10000, 10 ** 6, 128, 176, ib=10000)
    assert 0.4 * 10000 < a < 10000


def test_alt_impl_speedup():
    assert G["alt_baseline_ms"] / G["alt_fused_ms"] == pytest.approx(G["alt_speedup"], abs=0.05)
    assert G["alt_N"] / G["alt_L"] == G["alt_bin_width"]


def test_gb300_gamma_and_cop_budget():
    """Unit counts x clock: 152 x 64 x 2.07e9 ALU-pipe COP/s; against the
    measured BF16 peak the budget at D = 128 is under 3 COPs per score, so a
    compare-and-select per score (2 ALU COPs) already reaches the tensor time."""
    g_alu = RF.gb300_gamma("alu")
    assert g_alu == pytest.approx(152 * 64 * 2.07e9)
    assert RF.gb300_gamma("fma") == pytest.approx(2 * g_alu)
    budget = RF.cop_budget(128, g_alu, 1938.1e12)
    assert 2.5 < budget < 3.0


def test_report_picks_the_binding_roof():
    r = RF.report(1024, 10 ** 6, 128, 0.2e-3, 1938e12, 6686e9, RF.gb300_gamma(), 2.0,
                  260e6)
    assert r["binding"] == "tensor" and r["I_COP"] == pytest.approx(128.0)
    assert r["measured"] == pytest.approx(2 * 1024 * 10 ** 6 * 128 / 0.2e-3)
    r2 = RF.report(1024, 10 ** 6, 128, 0.2e-3, 1938e12, 6686e9, RF.gb300_gamma(), 4.0, 260e6)
    assert r2["binding"] == "cop"
