"""The paper's execution-time model (Sec. 4.5) reproduced from its own inputs:
every Table 6 cell from Table 4 (global words, operations) and Table 5 (STREAM,
DGEMM), and Table 4's arithmetic intensities. Two Table 6 cells (Xeon Phi, SSQ,
prisms) repeat the Xeon E5 SQS cells; the model gives 65.33 and 77.66 ns there."""
import json
import os

import pytest

from paper_1504_01023_gb300 import api, model

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "paper_time_model.json")
T = json.load(open(GOLDEN))
CASES = T["cases"]
# (machine, variant, case) cells printed with a copying slip, and the model's values
SLIPS = {("Phi5110P", "SSQ", "poisson_prism"): 65.33, ("Phi5110P", "SSQ", "convdiff_prism"): 77.66}


@pytest.mark.parametrize("machine", list(T["table6_ns"]))
@pytest.mark.parametrize("variant", ["QSS", "SQS", "SSQ"])
def test_table6_cells(machine, variant):
    bench = T["table5_benchmarks"][machine]
    for case, printed in zip(CASES, T["table6_ns"][machine][variant]):
        t = model.paper_time_bound_ns(T["table4_global_words"][case], T["table4_operations"][variant][case],
                                      bench["stream_gbs"], bench["dgemm_tflops"])
        if (machine, variant, case) in SLIPS:
            assert round(t, 2) == SLIPS[(machine, variant, case)]
            # the printed value is the Xeon E5 SQS cell of the same case
            assert printed == T["table6_ns"]["E5-2620x2"]["SQS"][CASES.index(case)]
        else:
            assert round(t, 2) == pytest.approx(printed, abs=0.006), (machine, variant, case, t, printed)


def test_table4_arithmetic_intensities():
    for variant, row in T["table4_arithmetic_intensity"].items():
        for case, printed in row.items():
            ai = model.arithmetic_intensity(T["table4_operations"][variant][case], T["table4_global_words"][case])
            assert round(ai) == printed, (variant, case, ai)


def test_table4_words_are_the_library_bytes():
    """The paper's global words (Table 4) times 8 are the library's algorithmic bytes
    for the same double-precision cases (TET4 and PRISM6; d^0 per point for
    Poisson, 20 coefficients per element for convection-diffusion)."""
    b = api.bytes_per_element
    got = {"poisson_tetra": b(api.TET, api.POISSON, api.QUAD_TET4, api.PER_QPOINT, api.FP64),
           "poisson_prism": b(api.PRISM, api.POISSON, api.QUAD_PRISM6, api.PER_QPOINT, api.FP64),
           "convdiff_tetra": b(api.TET, api.GENERIC, api.QUAD_TET4, api.PER_ELEMENT, api.FP64),
           "convdiff_prism": b(api.PRISM, api.GENERIC, api.QUAD_PRISM6, api.PER_ELEMENT, api.FP64)}
    for case, words in T["table4_global_words"].items():
        assert got[case] == 8 * words, (case, got[case])


def test_gb300_bound_of_the_headline():
    """The same model on this GPU's measured copy bandwidth: 256 B per element at
    6784.8 GB/s is 0.0377 ns, i.e. 26.5 Gelem/s, memory-bound (about 450
    float operations at ~70 TFlop/s take under 0.01 ns)."""
    t = model.time_bound_ns(256, 450, 6784.8, 70_000.0)
    assert t == pytest.approx(256 / 6784.8)
    assert 1.0 / t == pytest.approx(26.5, abs=0.05)
