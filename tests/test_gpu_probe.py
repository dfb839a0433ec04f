"""The unit-rate probe behind the filter's roofline (needs a GPU).

The roofline divides the filter's pair tests by a ceiling the probe measures:
population counts per clock per SM, 3-input logic operations per clock per
SM, and the filter's own k = 1 loop.  These tests hold the probe to what the
pipes can issue.  3-input logic runs on the integer ALU at no more than 64
results per clock per SM; the population count runs on the XU pipe at no more
than 16; the k = 1 loop spends 0.75 population counts per pair test, so it
cannot exceed 16 / 0.75.  The probe's SM clock (each SM's span of cycles over
the event-timed duration) must also agree with the clock the driver reports.
A probe that divided by something shorter than the SMs' real busy time would
report rates above these limits and a clock well below the driver's.
"""
import shutil
import subprocess

import pytest

pytestmark = pytest.mark.gpu

ALU_LOP3_PER_CLK_SM = 64.0
XU_POPC_PER_CLK_SM = 16.0


@pytest.fixture(scope="module")
def fp():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.init()
    from paper_1711_08475_gb300 import build
    build.build()
    import paper_1711_08475_gb300 as m
    return m


def test_probe_rates_within_pipe_limits(fp):
    lop3, popc, loop = (fp.fp_probe(k, 2000) for k in (1, 2, 3))
    for r in (lop3, popc, loop):
        assert r["sm_count"] > 0 and r["seconds"] > 0 and r["ops"] > 0
    assert 0.6 * ALU_LOP3_PER_CLK_SM <= lop3["ops_per_clk_per_sm"] <= 1.02 * ALU_LOP3_PER_CLK_SM, lop3
    assert 0.6 * XU_POPC_PER_CLK_SM <= popc["ops_per_clk_per_sm"] <= 1.02 * XU_POPC_PER_CLK_SM, popc
    assert loop["ops_per_clk_per_sm"] <= 1.02 * XU_POPC_PER_CLK_SM / 0.75, loop
    # the loop moves a quarter of its tests off the population-count pipe
    assert loop["ops_per_clk_per_sm"] > popc["ops_per_clk_per_sm"]


def test_probe_clock_agrees_with_driver(fp):
    import torch
    smi = shutil.which("nvidia-smi")
    if not smi:
        pytest.skip("nvidia-smi not available")
    out = subprocess.run([smi, "--query-gpu=clocks.max.sm", "--format=csv,noheader,nounits", "-i",
                          str(torch.cuda.current_device())], capture_output=True, text=True, timeout=60)
    if out.returncode != 0 or not out.stdout.strip():
        pytest.skip("nvidia-smi gave no clock")
    max_mhz = float(out.stdout.strip().splitlines()[0])
    r = fp.fp_probe(2, 4000)
    # a busy SM runs at (or, under a power cap, somewhat below) its maximum clock
    assert 0.7 * max_mhz <= r["sm_clock_mhz"] <= 1.03 * max_mhz, (r, max_mhz)
