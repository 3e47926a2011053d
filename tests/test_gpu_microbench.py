"""The peak microbenchmarks behind the bench's roofline: they run, and their rates are
plausible for the part (FP32 within [0.5, 1.2] of the nominal FMA rate at the device's
maximum clock; FP64 reductions above 1e9 per second)."""
from __future__ import annotations

import pytest

torch = pytest.importorskip("torch")

import paper_1612_09491_gb300 as pse  # noqa: E402

pytestmark = pytest.mark.gpu


def test_measured_peaks_are_plausible():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_1612_09491_gb300 import build
    build.build()
    p = pse.measure_peaks(fma_iters=1 << 14, red_per_thread=1024)
    props = torch.cuda.get_device_properties(0)
    clock_ghz = getattr(props, "clock_rate", 2070000) / 1e6 if hasattr(props, "clock_rate") else 2.07
    nominal = props.multi_processor_count * 128 * 2 * clock_ghz / 1e3
    assert 0.5 * nominal <= p["fp32_tflops"] <= 1.2 * nominal, (p, nominal)
    assert p["red_f64_per_s"] > 1e9, p
