"""Host-side logic of the benchmark (no GPU): the algorithmic byte and flop counts its roofline
fractions divide by, and the parsing of the clock samples it attaches to the JSON line."""
import bench


def test_algorithmic_bytes_match_the_stated_model():
    # 64^3 elements, N = 7: E = 262144, n^3 = 512, G = 449^3
    E, N, G = 64 ** 3, 7, 449 ** 3
    L = E * 512
    assert bench.algorithmic_bytes(E, N, G, "fp64") == 6 * 8 * L + 2 * 8 * G
    assert bench.algorithmic_bytes(E, N, G, "fp64_emu") == 6 * 8 * L + 2 * 8 * G
    assert bench.algorithmic_bytes(E, N, G, "fp32") == 6 * 4 * L + 2 * 4 * G
    assert bench.algorithmic_bytes(E, N, G, "bf16") == 6 * 2 * L + 2 * 4 * G
    assert bench.algorithmic_bytes(E, N, G, "fp32_otf") == 2 * 4 * G + 96 * E
    assert bench.algorithmic_bytes(E, N, G, "fp32_otf", kappa=True) == 2 * 4 * G + 96 * E + 4 * L
    # bytes per local DOF quoted in the design notes: 58.8 (FP64), 29.4 (FP32)
    assert abs(bench.algorithmic_bytes(E, N, G, "fp64") / L - 58.8) < 0.05
    assert abs(bench.algorithmic_bytes(E, N, G, "fp32") / L - 29.4) < 0.05


def test_flop_convention():
    # (12 n^4 + 15 n^3) per element: 111 per local DOF at N = 7
    assert bench.flops(1, 7) == 12 * 8 ** 4 + 15 * 8 ** 3
    assert abs(bench.flops(1, 7) / 512 - 111.0) < 1e-12


def test_clock_summary_flags_throttle_reasons():
    c = bench.ClockSampler()
    c.lines = ["0, 2070, 2070, 500.0, 0x0, Not Active, Not Active, Not Active, Not Active",
               "0, 1900, 2070, 1390.0, 0x4, Not Active, Not Active, Not Active, Active",
               "0, 2070, 2070, 700.0, 0x0, Not Active, Not Active, Not Active, Not Active",
               "garbage line"]
    s = c.summary()
    assert s["sm_mhz"] == 2070.0 and s["sm_max_mhz"] == 2070.0 and s["samples"] == 3
    assert s["reasons"] == ["sw_power_cap"]
    assert s["power_w_max"] == 1390.0
