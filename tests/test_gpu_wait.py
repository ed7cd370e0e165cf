"""Bounded host waits (SPGEMM_OPT_WAIT_LIMIT_MS): a wait that runs out
returns SPGEMM_ERR_TIMEOUT without touching the device work, which keeps
running and completes; the handle then serves correct calls again.  The
device is kept busy by a spin kernel that ends by itself (no fault, no
hang)."""
import pytest
import torch

import oracle
import paper_1804_00695_gb300 as sg
from paper_1804_00695_gb300 import inputs as I
from gpu_helpers import assert_matches, to_dev

pytestmark = pytest.mark.gpu


def _busy_ms(ms):
    """Queue about `ms` milliseconds of spinning on the current stream (a
    kernel that counts clock cycles and returns)."""
    props = torch.cuda.get_device_properties(torch.cuda.current_device())
    clock_khz = getattr(props, "clock_rate", 2_070_000)
    torch.cuda._sleep(int(ms * clock_khz))


def test_symbolic_wait_limit_times_out_then_recovers(cuda_lib):
    a, p, _ = I.galerkin_problem(12)
    A, P = to_dev(a), to_dev(p)
    h = sg.Handle()
    h.spgemm(A, P)                     # workspace sized: the timed call allocates nothing
    h.set_option(sg.OPT_WAIT_LIMIT_MS, 5)
    torch.cuda.synchronize()
    _busy_ms(300)                      # the symbolic call's kernels queue behind this
    with pytest.raises(sg.SpgemmError) as ei:
        h.symbolic(A, P)
    assert ei.value.status == 6        # SPGEMM_ERR_TIMEOUT
    torch.cuda.synchronize()           # the queued work completes
    # no valid symbolic phase on the handle now
    h.set_option(sg.OPT_WAIT_LIMIT_MS, 10_000)
    ref = oracle.spgemm(a, p)
    assert_matches(h.spgemm(A, P), ref, "f64")
    h.check()


def test_wait_limit_not_reached(cuda_lib):
    """A generous limit changes nothing: same product as without one."""
    a, p, r = I.galerkin_problem(16)
    h = sg.Handle()
    h.set_option(sg.OPT_WAIT_LIMIT_MS, 60_000)
    ap = h.spgemm(to_dev(a), to_dev(p))
    assert_matches(ap, oracle.spgemm(a, p), "f64")


def test_wait_limit_rejects_negative(cuda_lib):
    h = sg.Handle()
    with pytest.raises(sg.SpgemmError) as ei:
        h.set_option(sg.OPT_WAIT_LIMIT_MS, -1)
    assert ei.value.status == 1
