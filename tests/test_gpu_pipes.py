"""The SM pipe probes behind the CUDA-core rooflines (ap_pipe_rate): each
measured rate must sit near what one SM of this GPU can issue -- 128 FP32
FMA lanes, a MUFU unit an eighth to a quarter of that -- so that a probe the
compiler optimised away (a reported rate far above the hardware's) fails."""
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ap():
    import paper_2009_04755_gb300 as ap
    ap.lib()
    return ap


def test_pipe_rates_are_physical(ap):
    b = ap.binding
    ffma = b.pipe_rate(b.PIPE_FMA)
    assert 100 <= ffma["per_clk_per_sm"] <= 130
    assert 500 <= ffma["sm_mhz"] <= 2500
    ffma2 = b.pipe_rate(b.PIPE_FMA2)
    assert 100 <= ffma2["per_clk_per_sm"] <= 260
    for pipe in (b.PIPE_EX2, b.PIPE_RCP):
        r = b.pipe_rate(pipe)
        assert 8 <= r["per_clk_per_sm"] <= 64, (pipe, r)
        # results per second agree with per clock x SMs x clock
        n_sm = torch.cuda.get_device_properties(0).multi_processor_count
        est = r["per_clk_per_sm"] * n_sm * r["sm_mhz"] * 1e6
        assert 0.7 * est <= r["per_s"] <= 1.3 * est


def test_pipe_rate_rejects_unknown_pipe(ap):
    import ctypes
    a, b_, c = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    assert ap.lib().ap_pipe_rate(7, ctypes.byref(a), ctypes.byref(b_), ctypes.byref(c)) == 1
