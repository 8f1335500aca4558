"""The split 16-bit precisions on the tensor cores (tcgen05.mma with FP32
accumulation in tensor memory): one axis pass of the batched 3-D DFT against
numpy's FFT, and L[g] against the CPU oracle.

Stated bounds.  A split operand x = x_hi + x_lo (16-bit parts) leaves
~2^-16 (BF16, 8-bit significands) or ~2^-22 (FP16, 11 bits, with the
pencil's power-of-two scale) of |x|, and the dropped product x_lo W_lo is
of the same order; the FP32 accumulation of the 2N products of an output
adds ~2^-24 sqrt(2N) of their size, which is the larger term for FP16.  So a
transform carries a relative error u_eff = 2^-16 (BF16) or 2^-21 (FP16, the
accumulation floor) of the data's size (measured: 0.06 and 0.5-0.6 of the
one-pass bound below).  For one axis pass the bound is 4 u_eff sqrt(N)
max|x| on max|y - y_ref|.  For L[g] the FFT form's error grows with the ratio
r = g/M it transforms (Sec. 3.3): the bound is 4 u_eff rms(r), as for the
other reduced precisions."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle.linearized import Tables, apply_linearized
from paper_2503_09580_gb300 import lbo, workloads

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
U_EFF = {"bf16_split": 2.0 ** -16, "fp16_split": 2.0 ** -21}


def numpy_axis_dft(x, axis, inverse):
    """The pass's definition: forward sum_j x_j exp(-2 pi i q (j - N/2)/N)
    (centred j -> cyclic q), inverse the conjugate kernel, unnormalised."""
    n = x.shape[axis]
    sign = np.where(np.arange(n) % 2 == 0, 1.0, -1.0)
    shape = [1] * x.ndim
    shape[axis] = n
    s = sign.reshape(shape)
    if inverse:
        return n * np.fft.ifft(x * s, axis=axis)
    return np.fft.fft(x, axis=axis) * s


@pytest.mark.parametrize("precision", ["bf16_split", "fp16_split"])
@pytest.mark.parametrize("n", [16, 32, 64])
def test_axis_pass_matches_numpy(precision, n):
    rng = np.random.default_rng(n)
    batch = 2
    x = rng.standard_normal((batch, n, n, n)) + 1j * rng.standard_normal((batch, n, n, n))
    x[0] *= 1e3  # instances of different sizes: the split is per pencil
    xt = torch.from_numpy(np.stack([x.real, x.imag], -1).astype(np.float32)).to(DEV).contiguous()
    for axis in (1, 2, 3):
        for inverse in (0, 1):
            out = torch.empty_like(xt)
            lbo.dft_axis_tensor(n, precision, inverse, axis, xt, out)
            got = out.cpu().numpy().astype(np.float64)
            got = got[..., 0] + 1j * got[..., 1]
            xin = xt.cpu().numpy().astype(np.float64)
            ref = numpy_axis_dft(xin[..., 0] + 1j * xin[..., 1], axis, inverse)
            for b in range(batch):
                err = np.abs(got[b] - ref[b]).max()
                bound = 4 * U_EFF[precision] * np.sqrt(n) * np.abs(xin[b]).max()
                print("%s n=%d axis %d inv %d: err/bound %.3f" % (precision, n, axis, inverse, err / bound))
                assert err <= bound


def rms_r(params, g, n, L, eps=1e-9):
    a = workloads.velocity_axis(n, L)
    out = []
    for b in range(params.shape[0]):
        rho, u1, u2, u3, th = params[b]
        d2 = (a[:, None, None] - u1) ** 2 + (a[None, :, None] - u2) ** 2 + (a[None, None, :] - u3) ** 2
        M = rho * (2 * np.pi * th) ** -1.5 * np.exp(-d2 / (2 * th))
        keep = d2 / (2 * th) <= np.log(1 / eps) - 1.5 * np.log(2 * np.pi * th)
        r = np.where(keep, g[b] / M, 0.0)
        out.append(np.sqrt(np.mean(r * r)))
    return np.array(out)


@pytest.mark.parametrize("precision", ["bf16_split", "fp16_split"])
@pytest.mark.parametrize("n,noise", [(16, 0.0), (32, 0.0), (32, 1e-3)])
def test_linearized_split_precisions_within_stated_bound(precision, n, noise):
    L = 8.0
    params, g = workloads.batched_instances(n, L, batch=3, seed=61, noise=noise)
    tp, tg = torch.from_numpy(params).to(DEV), torch.from_numpy(g).to(DEV)
    out = torch.empty_like(tg)
    plan = lbo.Plan(n, L, 0.5, n, precision=precision)
    plan.apply_linearized(tp, tg, out)
    plan.sync()
    got = out.cpu().numpy()
    ref = apply_linearized(Tables(n, L, 0.5, n), params, g)
    bound = 4 * U_EFF[precision] * rms_r(params, g, n, L)
    for b in range(3):
        err = np.abs(got[b] - ref[b]).max() / np.abs(ref[b]).max()
        print("%s n=%d noise %g: err %.3e bound %.3e" % (precision, n, noise, err, bound[b]))
        assert err <= bound[b]
    # the cached Maxwellian factors give the same result
    plan.cache_maxwellians(tp)
    out2 = torch.empty_like(tg)
    plan.apply_linearized(tp, tg, out2)
    plan.sync()
    assert np.array_equal(out2.cpu().numpy(), got)


def test_split_precision_n64_against_oracle_one_instance():
    n, L = 64, 8.0
    params, g = workloads.batched_instances(n, L, batch=1, seed=62, noise=0.0)
    tp, tg = torch.from_numpy(params).to(DEV), torch.from_numpy(g).to(DEV)
    ref = apply_linearized(Tables(n, L, 1.0, n), params, g)
    for precision in ("bf16_split", "fp16_split"):
        out = torch.empty_like(tg)
        plan = lbo.Plan(n, L, 1.0, n, precision=precision)
        plan.apply_linearized(tp, tg, out)
        plan.sync()
        err = np.abs(out.cpu().numpy()[0] - ref[0]).max() / np.abs(ref[0]).max()
        bound = 4 * U_EFF[precision] * rms_r(params, g, n, L)[0]
        print("%s n=64: err %.3e bound %.3e" % (precision, err, bound))
        assert err <= bound


def test_split_precision_refuses_unbuilt_sizes_and_quadratic():
    n, L = 24, 8.0
    params, g = workloads.batched_instances(n, L, batch=1, seed=63, noise=0.0)
    tp, tg = torch.from_numpy(params).to(DEV), torch.from_numpy(g).to(DEV)
    plan = lbo.Plan(n, L, 0.5, n, precision="bf16_split")
    with pytest.raises(lbo.LboError) as ei:
        plan.apply_linearized(tp, tg, torch.empty_like(tg))
    assert ei.value.status == 7
    n, L = 32, 8.0
    f = torch.from_numpy(workloads.batched_instances(n, L, batch=1, seed=64, noise=0.0)[1]).to(DEV)
    plan = lbo.Plan(n, L, 0.5, n, precision="fp16_split")
    with pytest.raises(lbo.LboError) as ei:
        plan.apply_quadratic(f, torch.empty_like(f))
    assert ei.value.status == 7
