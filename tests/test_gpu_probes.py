"""The arithmetic-rate probes (itp_peak_probe) that give the ALU and tensor
rooflines their denominators: each returns a finite, positive rate in the
range a GB300 can deliver (nominal: FP32 ~80 TFLOP/s, FP64 ~1.2 TFLOP/s,
TF32 tensor ~1.1 PFLOP/s dense), and the tensor-core probe's bounded wait
does not expire."""
import math

import pytest

pytestmark = pytest.mark.gpu

import paper_0809_3739_gb300 as P  # noqa: E402


@pytest.mark.parametrize("kind,lo,hi", [("ffma", 10.0, 200.0), ("ffma2", 10.0, 400.0),
                                        ("dfma", 0.2, 100.0), ("tf32_mma", 100.0, 3000.0)])
def test_peak_probe_rates_are_plausible(kind, lo, hi):
    t, ms = P.itp_peak_probe(kind)
    print(f"[probe] {kind}: {t:.2f} TFLOP/s, {ms:.2f} ms per launch", flush=True)
    assert math.isfinite(t) and lo < t < hi
    assert ms > 0


def test_peak_probe_rejects_unknown_kind():
    with pytest.raises(P.ItpError) as ei:
        P.itp_peak_probe(7)
    assert ei.value.code == P.itp.ITP_ERR_ARG
