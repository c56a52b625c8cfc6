"""Gaussian beam convolution (Sec. 4.11, irt_beam_convolve) against the FP64
oracle: float and double, several beam widths, edges, in-place output and
argument checks."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

import oracle  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2607_01338_b300  # noqa: F401


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
@pytest.mark.parametrize("fwhm,shape", [(2.0, (3, 40, 50)), (3.3, (2, 17, 64)),
                                        (7.0, (1, 64, 33)), (30.0, (1, 5, 300))])
def test_beam_against_oracle(fwhm, shape, dtype):
    import paper_2607_01338_b300 as irt
    rng = np.random.default_rng(int(fwhm * 10) + shape[1])
    x = torch.from_numpy(rng.uniform(0.0, 5.0, shape)).to(dtype).cuda()
    got = irt.beam_convolve(x, fwhm).double().cpu().numpy()
    exp = oracle.beam_convolve(x.double().cpu().numpy(), fwhm)
    tol = 2e-6 if dtype == torch.float32 else 1e-13
    np.testing.assert_allclose(got, exp, rtol=tol, atol=tol * float(np.abs(exp).max()))


def test_beam_in_place_and_checks():
    import paper_2607_01338_b300 as irt
    from paper_2607_01338_b300 import binding as B
    x = torch.rand((2, 30, 40), device="cuda")
    exp = oracle.beam_convolve(x.double().cpu().numpy(), 4.0)
    irt.beam_convolve(x, 4.0, out=x)
    np.testing.assert_allclose(x.double().cpu().numpy(), exp, rtol=2e-6, atol=2e-6)
    with pytest.raises(B.IrtError, match="taps"):
        irt.beam_convolve(x, 100.0)
    with pytest.raises(B.IrtError, match="FWHM"):
        irt.beam_convolve(x, 0.0)
    with pytest.raises(B.IrtError, match="separate"):
        B.irt_beam_convolve(x.data_ptr(), B.IRT_F32, 2, 30, 40, 3.0, x.data_ptr(), x.data_ptr())
