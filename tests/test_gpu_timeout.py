"""Failure detection without a GPU fault: every barrier wait of the tensor-core kernels is
bounded, and a wait that runs out makes the kernel drain its own copies and MMAs, free its
tensor memory, set the device error word and return.  The wait budget is a tuning knob
(rgeo_tuning.wait_limit), so the test makes the waits give up at once; rgeo_sync must then
report RGEO_ETIMEOUT, and the context must stay usable: the same calls with the default
budget succeed and give the right answer."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rg():
    import torch
    import paper_2005_05386_gb300 as rg
    torch.cuda.set_device(0)
    return rg


def _gemm(rg, A, B, C):
    M, K = A.shape
    N = B.shape[0]
    rg.rgeo_gemm_bf16(A.data_ptr(), B.data_ptr(), M, N, K, 1, None, 0, C.data_ptr(), N, None, 0)


def test_waits_that_run_out_report_timeout_and_leave_the_context_usable(rg):
    import torch
    g = torch.Generator(device="cuda").manual_seed(3)
    A = (torch.rand((128, 512), generator=g, device="cuda") - 0.5).to(torch.bfloat16)
    B = (torch.rand((256, 512), generator=g, device="cuda") - 0.5).to(torch.bfloat16)
    C = torch.zeros((128, 256), device="cuda")
    ex = rg.Expmap(max_batch=256, seed=5)
    X = torch.rand((128, 7), generator=g, device="cuda") * 2 - 1
    T = torch.rand((128, 6), generator=g, device="cuda") - 0.5
    p0 = ex.get_params()
    rg.rgeo_sync()
    try:
        rg.rgeo_set_tuning(wait_limit=-1)
        assert rg.rgeo_get_tuning()["wait_limit"] == -1
        _gemm(rg, A, B, C)  # 8 K-stages: the wait for the first stage's MMAs gives up
        with pytest.raises(rg.RgeoError) as e:
            rg.rgeo_sync()
        assert e.value.status == rg.RGEO_ETIMEOUT, e.value
        ex.forward(X)  # persistent inference: the producer's and the MMA issuer's waits give up
        with pytest.raises(rg.RgeoError) as e:
            rg.rgeo_sync()
        assert e.value.status == rg.RGEO_ETIMEOUT, e.value
        # fused training step: the first product's stage wait gives up; the Adam kernel then
        # leaves the parameters alone
        ex.train_step(X, T, 1e-3)
        with pytest.raises(rg.RgeoError) as e:
            rg.rgeo_sync()
        assert e.value.status == rg.RGEO_ETIMEOUT, e.value
        assert np.array_equal(ex.get_params(), p0)
    finally:
        rg.rgeo_set_tuning()
    assert rg.rgeo_get_tuning()["wait_limit"] == 0
    rg.rgeo_sync()  # the error word was cleared by the report
    C.zero_()
    _gemm(rg, A, B, C)
    Y = ex.forward(X)
    G, L = ex.gradients(X, T)
    rg.rgeo_sync()
    torch.testing.assert_close(C, A.float() @ B.float().T, rtol=1e-5, atol=1e-4 * 512 ** 0.5)
    assert np.isfinite(Y.cpu().numpy()).all()
    assert np.isfinite(G.cpu().numpy()).all() and L.item() > 0
