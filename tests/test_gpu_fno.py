"""GPU FNO kernels against the FP64 reference (oracle/fno_ref.py): forward,
loss and every parameter gradient at BF16-operand / FP32-accumulate accuracy,
and training through the library's own Adam step."""
import numpy as np
import pytest

from oracle import fno_ref as F
from tests.gpu_helpers import need_gpu

pytestmark = pytest.mark.gpu


def _model(cfgref, batch, seed=3):
    from paper_1007_3470_gb300.fno import Fno, FnoConfig
    cfg = FnoConfig(grid=cfgref.L, width=cfgref.C, modes=cfgref.M, layers=cfgref.layers, in_ch=cfgref.in_ch,
                    proj=cfgref.P, out_ch=cfgref.out)
    m = Fno(cfg, max_batch=batch, train=True, seed=None)
    p = F.init_params(cfgref, seed)
    rng = np.random.default_rng(seed)
    for k in p:                      # non-zero biases so that every path is exercised
        if k.startswith(("b", "c")):
            p[k] = 0.1 * rng.standard_normal(p[k].shape)
    vec = F.pack(cfgref, p).astype(np.float32)
    m.set_params(vec)
    return m, F.unpack(cfgref, vec.astype(np.float64))


def _data(cfgref, B, seed=5):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((B, cfgref.L, cfgref.in_ch))
    Y = rng.standard_normal((B, cfgref.L, cfgref.out))
    return X, Y


def _rel(a, b):
    return float(np.linalg.norm(np.ravel(a - b)) / np.linalg.norm(np.ravel(b)))


@pytest.mark.parametrize("cfgref", [F.Config(L=64, C=16, M=8, layers=2, in_ch=7, P=32, out=2),
                                    F.Config(L=256, C=64, M=32, layers=4, in_ch=7, P=128, out=2)])
def test_forward_matches_reference(cfgref):
    torch = need_gpu()
    m, p = _model(cfgref, 3)
    X, _ = _data(cfgref, 3)
    out = m.forward(torch.from_numpy(X.astype(np.float32))).cpu().numpy()
    ref = F.forward(cfgref, p, X)
    assert _rel(out, ref) < 3e-2
    m.close()


def test_gradients_match_reference():
    torch = need_gpu()
    cfgref = F.Config(L=64, C=16, M=8, layers=2, in_ch=7, P=32, out=2)
    m, p = _model(cfgref, 4)
    X, Y = _data(cfgref, 4)
    loss, g = m.loss_grad(torch.from_numpy(X.astype(np.float32)), torch.from_numpy(Y.astype(np.float32)))
    lref, gref = F.loss_and_grad(cfgref, p, X, Y)
    assert abs(loss - lref) < 2e-2 * lref
    gg = F.unpack(cfgref, g.cpu().numpy().astype(np.float64))
    for name, _ in cfgref.shapes():
        assert _rel(gg[name], gref[name]) < 0.1, name
    a, b = g.cpu().numpy().astype(np.float64), F.pack(cfgref, gref)
    assert float(a @ b / (np.linalg.norm(a) * np.linalg.norm(b))) > 0.995


def test_adam_training_reduces_loss():
    torch = need_gpu()
    cfgref = F.Config(L=64, C=16, M=8, layers=2, in_ch=7, P=32, out=2)
    m, _ = _model(cfgref, 32)
    rng = np.random.default_rng(1)
    X = rng.standard_normal((32, 64, 7)).astype(np.float32)
    # a smooth target that the model can represent: a low-pass of two input channels
    Y = np.stack([np.cumsum(X[..., 0], axis=1) / 8, X[..., 1] * 0.5], axis=-1).astype(np.float32)
    xd, yd = torch.from_numpy(X).cuda(), torch.from_numpy(Y).cuda()
    torch.cuda.synchronize()
    first = m.train_step(xd, yd, 3e-3)
    for _ in range(150):
        last = m.train_step(xd, yd, 3e-3)
    assert last < 0.5 * first, (first, last)
    m.close()


def test_tensor_core_gemms_forward_and_gradients():
    """With the tcgen05 engine, rows >= 8192 with widths of 64 and 128 take
    the tensor-core GEMMs (operands in shared memory, accumulators in tensor
    memory): the pointwise layers (K = N = 64, B plain and transposed in the
    backward pass), the projection (N = 128) and its backward product
    (K = 128).  64 x 129 rows leave the last 128-row tile ragged.  Same bounds
    as the mma.sync path above, and no bounded wait runs out."""
    torch = need_gpu()
    cfgref = F.Config(L=64, C=64, M=8, layers=2, in_ch=7, P=128, out=2)
    B = 129
    from paper_1007_3470_gb300.fno import HFS_FNO_GEMM_TCGEN05
    m, p = _model(cfgref, B)
    m.set_gemm_engine(HFS_FNO_GEMM_TCGEN05)
    X, Y = _data(cfgref, B)
    out = m.forward(torch.from_numpy(X.astype(np.float32))).cpu().numpy()
    assert _rel(out, F.forward(cfgref, p, X)) < 3e-2
    loss, g = m.loss_grad(torch.from_numpy(X.astype(np.float32)), torch.from_numpy(Y.astype(np.float32)))
    lref, gref = F.loss_and_grad(cfgref, p, X, Y)
    assert abs(loss - lref) < 2e-2 * lref
    gg = F.unpack(cfgref, g.cpu().numpy().astype(np.float64))
    for name, _ in cfgref.shapes():
        assert _rel(gg[name], gref[name]) < 0.1, name
    a, b = g.cpu().numpy().astype(np.float64), F.pack(cfgref, gref)
    assert float(a @ b / (np.linalg.norm(a) * np.linalg.norm(b))) > 0.995
    assert m.status() == 0
    m.close()
