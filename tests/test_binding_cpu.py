"""Host-side argument checks of the Python binding: wrong devices, dtypes and
shapes are refused before anything reaches the library (no GPU needed)."""
import pytest
import torch

from paper_2401_09721_gb300 import build


@pytest.fixture(scope="module")
def F():
    build.build()
    from paper_2401_09721_gb300 import fgbd
    return fgbd


def test_inputs_must_be_cuda_int32_n_by_3(F):
    with pytest.raises(TypeError):
        F.fgbd_build_graph(None, torch.zeros((4, 3), dtype=torch.float32))
    with pytest.raises(ValueError, match="CUDA"):
        F.fgbd_build_graph(None, torch.zeros((4, 3), dtype=torch.int32))
    with pytest.raises(ValueError, match="CUDA"):
        F.fgbd_estimate_noise(None, torch.zeros((4, 3), dtype=torch.uint8))


def test_differentiable_filter_takes_float32(F):
    z8 = torch.zeros((4, 3), dtype=torch.uint8)
    z32 = torch.zeros((4, 3), dtype=torch.float32)
    with pytest.raises(TypeError):
        F.fgbd_filter_forward(None, z8, 1, 0.5, 0.0, 1, z32, 4)
    with pytest.raises(ValueError, match="CUDA"):
        F.fgbd_filter_forward(None, z32, 1, 0.5, 0.0, 1, z32, 4)


def test_status_names_and_constants(F):
    assert F.STATUS[7] == "FGBD_ENOTIMPL"
    err = F.FgbdError(7, "fgbd_ctx_create")
    assert err.status == 7 and "FGBD_ENOTIMPL" in str(err)
    assert F.PATCH_DIM == 21 and F.PATCH_DIM_MAX == 3 * (6 * F.MAX_WINDOW + 1)
