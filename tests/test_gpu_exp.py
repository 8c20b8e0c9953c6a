"""The FP64 exp of the rate evaluation (Tang's table-driven method) on the
GPU: within 0.6 ulp of the exact value (mpmath) and within 1 ulp of the
CUDA library exp."""
import mpmath
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_exp_tang_error_bound():
    import ctypes as C

    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2312_02836_gb300 import _abi
    lib = _abi.load()
    rng = np.random.default_rng(11)
    x = np.concatenate([rng.uniform(-700, 700, 4000), rng.uniform(-1, 1, 4000),
                        rng.normal(0, 60, 4000),
                        np.array([0.0, -0.0, 700.0, -700.0, 709.5, -720.0, -745.5,
                                  np.inf, -np.inf, np.nan])])
    dev = torch.device("cuda")
    xd = torch.from_numpy(x).to(dev)
    yt = torch.empty_like(xd)
    yl = torch.empty_like(xd)
    assert lib.nb_exp_eval(xd.data_ptr(), yt.data_ptr(), yl.data_ptr(), x.size,
                           C.c_void_p(torch.cuda.current_stream().cuda_stream)) == 0
    torch.cuda.synchronize()
    yt, yl = yt.cpu().numpy(), yl.cpu().numpy()
    fin = np.isfinite(x) & (np.abs(x) <= 700)
    ulp = np.spacing(np.abs(yl[fin]))
    assert np.all(np.abs(yt[fin] - yl[fin]) <= ulp)
    mpmath.mp.prec = 120
    worst = 0.0
    for xi, yi in zip(x[fin][::7], yt[fin][::7]):
        e = mpmath.e ** mpmath.mpf(float(xi))
        worst = max(worst, float(abs(mpmath.mpf(float(yi)) - e) / np.spacing(float(e))))
    assert worst <= 0.6, worst
    # outside |x| <= 700 the library exp is used as is
    out = ~fin
    assert np.array_equal(yt[out], yl[out], equal_nan=True)
