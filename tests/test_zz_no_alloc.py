"""The allocation-free projection entry point (ldgmg_project_kernel_noalloc).

It serves callers that must not call cudaMalloc (device memory owned by
another allocator, or loops that cannot take cudaMalloc's implicit
synchronisation).  Its scratch is a fixed device array inside the library, so
this test checks, through the C-ABI, that two calls in a row (different sizes
and data, sharing that array) give the same result as the allocating
ldgmg_project_kernel, and that oversized inputs are refused.  It lives in its
own file, collected last, and needs nothing from the other tests.
"""
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_project_kernel_noalloc_matches_allocating_version():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2412_12506_gb300 import ldgmg
    gen = torch.Generator(device="cuda").manual_seed(11)
    for d, n, p in [(3, 20, 3), (2, 37, 2)]:          # two calls in a row, different sizes
        op = ldgmg.Operator(d, n, p)
        v = torch.randn(op.size, dtype=torch.float64, device="cuda", generator=gen)
        ref = op.project_kernel(v.clone())
        got = ldgmg.project_kernel_noalloc(v.clone(), op.N, op.b)
        torch.cuda.synchronize()
        err = float((got - ref).abs().max() / ref.abs().max())
        assert err < 1e-14, err
        # the constant mode is gone: mode-0 coefficients have zero mean
        assert abs(float(got[0::op.b].mean())) < 1e-13


def test_project_kernel_noalloc_rejects_oversized_input():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2412_12506_gb300 import ldgmg
    v = torch.zeros(8, dtype=torch.float64, device="cuda")
    with pytest.raises(ldgmg.LdgmgError) as e:
        ldgmg.project_kernel_noalloc(v, ldgmg.NOALLOC_MAX_ELEMENTS + 1, 1)
    assert e.value.status == ldgmg.EINVAL and "exceeds the maximum" in str(e.value)
