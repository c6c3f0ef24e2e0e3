"""The Python binding refuses tensors the kernels cannot address (host tensors for
the device entry points, device tensors where host memory is expected) with a
ValueError, before any call into the library: no CPU fallback, and no host pointer
ever reaches a kernel.  Runs without a GPU."""
import pytest
import torch


@pytest.fixture(scope="module")
def mm(libpath):
    import paper_2305_00332_gb300 as pkg
    return pkg


def test_device_entry_points_refuse_host_tensors(mm):
    y = torch.zeros(100, dtype=torch.float32)
    for call in (lambda: mm.minmaxlttb(y, 10, 4), lambda: mm.minmax_preselect(y, 10, 4),
                 lambda: mm.m4(y, 12), lambda: mm.lttb(y, 10), lambda: mm.check_series(y),
                 lambda: mm.raster(y, (0, 99, -1, 1), 8, 8),
                 lambda: mm.Batch([{"y": y, "n_out": 10}])):
        with pytest.raises(ValueError, match="CUDA"):
            call()


def test_images_and_workspaces_must_be_device_tensors(mm):
    with pytest.raises(ValueError, match="CUDA"):
        mm.intensity(torch.zeros((4, 4), dtype=torch.int32))
    img = torch.zeros((4, 4), dtype=torch.uint8)
    with pytest.raises(ValueError, match="CUDA"):
        mm.visual_counts(img, img)
    ws = torch.zeros(256, dtype=torch.uint8)
    with pytest.raises(ValueError, match="CUDA"):
        mm.workspace_status(ws)
    with pytest.raises(ValueError, match="CUDA"):
        mm.diag_wait_timeout(mm.DIAG_FUSED_BARRIER, ws)


def test_shape_checks(mm):
    with pytest.raises(ValueError, match="1-D"):
        mm.minmaxlttb(torch.zeros((3, 3)), 5, 4)
