"""The error bound behind the chosen form's tensor-core translations, on
the CPU: a value split into bf16 hi + lo (hi = bf16(v), lo = bf16(v - hi))
and the three products hi*hi + hi*lo + lo*hi accumulated in FP32 reproduce
a complex matrix-vector product of the translations' sizes to a few 1e-6
relative (bf16 keeps 8 significant bits, so hi + lo keeps about 16: a
representation error up to 2^-17 per factor; the dropped lo*lo term and the
FP32 accumulation add less), far below the 1e-4 accuracy of the method;
one bf16 product alone would be ~1e-3."""
import numpy as np
import pytest


def _bf16(x):
    """Round float32 to bfloat16 (nearest, ties to even), returned as float32."""
    b = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    r = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return r.astype(np.uint32).view(np.float32)


def _split(v):
    hi = _bf16(v)
    lo = _bf16(v.astype(np.float32) - hi)
    return hi, lo


@pytest.mark.parametrize("T", [64, 135, 342])
def test_split_bf16_three_products(T):
    rng = np.random.default_rng(T)
    A = (rng.standard_normal((T, T)) + 1j * rng.standard_normal((T, T))) / np.sqrt(T)
    x = rng.standard_normal(T) + 1j * rng.standard_normal(T)
    exact = A @ x
    # the stacked real form the kernel uses: [Ar; Ai] times [xr, xi]
    Ar, Ai = A.real.astype(np.float32), A.imag.astype(np.float32)
    xr, xi = x.real.astype(np.float32), x.imag.astype(np.float32)
    (Arh, Arl), (Aih, Ail) = _split(Ar), _split(Ai)
    (xrh, xrl), (xih, xil) = _split(xr), _split(xi)

    def mm(a_h, a_l, b_h, b_l):
        f = np.float32
        return (a_h.astype(f) @ b_h.astype(f) + a_h.astype(f) @ b_l.astype(f) + a_l.astype(f) @ b_h.astype(f))

    re = mm(Arh, Arl, xrh, xrl) - mm(Aih, Ail, xih, xil)
    im = mm(Arh, Arl, xih, xil) + mm(Aih, Ail, xrh, xrl)
    got = re.astype(np.float64) + 1j * im.astype(np.float64)
    err = np.linalg.norm(got - exact) / np.linalg.norm(exact)
    assert err < 1e-5
    one = (Arh @ xrh - Aih @ xih).astype(np.float64) + 1j * (Arh @ xih + Aih @ xrh).astype(np.float64)
    err1 = np.linalg.norm(one - exact) / np.linalg.norm(exact)
    assert 1e-4 < err1 < 1e-2
