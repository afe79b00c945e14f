"""Device-side error reporting through the C ABI (cfs_stream_status).

A kernel whose bounded wait runs out sets a bit in the device's error word;
the flag is made here from the host (cfs_debug_raise_device_error), so no
kernel has to time out.  Checks that the status call reports it once, that
the sampler's checkpoint call reports the same word, and that ordinary work
reports OK."""
import numpy as np
import pytest

from paper_2606_02226_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _cfs():
    from paper_2606_02226_gb300 import cfs
    return cfs


def _small_render(torch, stream=None):
    cfs = _cfs()
    wl = W.square_render(n_points=4096, iters=40, burn_in=20, W=64)
    t = cfs.alloc_target(wl.targets[0])
    cfs.render(cfs.System(wl.jobs[0].system), cfs.Chain(wl.chain, 2), wl.targets, [t],
               n_points=4096, iters=40, burn_in=20, stream=stream)
    return t


def test_status_ok_after_ordinary_work(torch_cuda):
    cfs = _cfs()
    cfs.stream_status()                      # clears anything earlier tests left
    t = _small_render(torch_cuda)
    cfs.stream_status()
    assert int(t.view(torch_cuda.int32).sum().item()) == 4096 * 20


def test_timeout_flag_is_reported_once(torch_cuda):
    cfs = _cfs()
    cfs.stream_status()
    cfs.debug_raise_device_error(cfs.DEVICE_ERR_TC_TIMEOUT)
    with pytest.raises(cfs.CfsError) as e:
        cfs.stream_status()
    assert e.value.status == 6 and "timed out" in str(e.value)
    cfs.stream_status()                      # reported once, then cleared


def test_timeout_flag_on_a_torch_stream(torch_cuda):
    torch = torch_cuda
    cfs = _cfs()
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        _small_render(torch, stream=s)
    cfs.debug_raise_device_error(cfs.DEVICE_ERR_TC_TIMEOUT)
    with pytest.raises(cfs.CfsError) as e:
        cfs.stream_status(s)
    assert e.value.status == 6
    cfs.stream_status(s)


def test_sampler_checkpoint_reports_the_same_word(torch_cuda):
    cfs = _cfs()
    sm = cfs.Sampler(seed=1)
    cfs.stream_status()
    cfs.debug_raise_device_error(cfs.DEVICE_ERR_TC_TIMEOUT)
    with pytest.raises(cfs.CfsError) as e:
        sm.get_params()
    assert e.value.status == 6
    cfs.stream_status()                      # already reported by the checkpoint
    w, _, _, _ = sm.get_params()
    assert np.isfinite(w).all()
