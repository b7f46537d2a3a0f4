"""The FP64 throughput probes behind the roofline's denominator: the FMA-pipe probe agrees with
the figure derived from the unit counts and the clock (152 SMs x 2 DFMA/clk x 2 flop x clock),
and the FP64 tensor-core (DMMA) probe returns a finite positive rate."""
import math

import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_fp64_probes(mdp):
    dfma = mdp.probe_fp64_gflops()
    dmma = mdp.probe_dmma_gflops()
    assert math.isfinite(dfma) and math.isfinite(dmma)
    derived = 152 * 2 * 2 * 2.070
    assert 0.5 * derived < dfma < 1.2 * derived, dfma
    assert 0.0 < dmma < 1e5, dmma
