"""Failure detection on the GPU without a fault: the persistent PCG's grid
barrier has a bounded spin; a diagnostic launch that waits for a block that
does not exist must come back with OSMPM_E_TIMEOUT, and the CUDA context
must stay usable afterwards."""
import numpy as np
import pytest

from paper_2605_09097_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def test_device_wait_times_out_and_context_survives():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_09097_gb300 import build
    build.build()
    from paper_2605_09097_gb300 import osmpm
    st = osmpm.osmpm_check_wait_timeout(torch.cuda.current_stream().cuda_stream)
    assert st == osmpm.OSMPM_E_TIMEOUT, osmpm.osmpm_last_error()
    spec = W.block(2, n_cells=(3, 3), dx=0.1, gravity=(0.0, -9.81))
    dom = osmpm.Domain(spec)
    dom.step(0.01)
    x = dom.get_particles()[0]
    assert np.all(np.isfinite(x))
