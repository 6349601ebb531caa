"""The allocation-free projection entry point (ldgmg_project_kernel_noalloc).

It serves callers that must not call cudaMalloc (device memory owned by
another allocator, or loops that cannot take cudaMalloc's implicit
synchronisation).  Its scratch is a fixed device array inside the library, so
this test checks, through the C-ABI, that calls in a row (different sizes and
data, sharing that array) give the same result as the allocating
ldgmg_project_kernel -- scalar vectors in one call, Stokes vectors in one call
per field -- that the largest admissible size and a size one past a full
scratch chunk are handled, and that oversized or too-short inputs are refused.
It lives in its own file, collected last, and needs nothing from the other
tests.
"""
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2412_12506_gb300 import ldgmg
    return ldgmg


def test_project_kernel_noalloc_matches_allocating_version(lib):
    gen = torch.Generator(device="cuda").manual_seed(11)
    for d, n, p in [(3, 20, 3), (2, 37, 2)]:          # two calls in a row, different sizes
        op = lib.Operator(d, n, p)
        v = torch.randn(op.size, dtype=torch.float64, device="cuda", generator=gen)
        ref = op.project_kernel(v.clone())
        got = lib.project_kernel_noalloc(v.clone(), op.N, op.b)
        torch.cuda.synchronize()
        err = float((got - ref).abs().max() / ref.abs().max())
        assert err < 1e-14, err
        # the constant mode is gone: mode-0 coefficients have zero mean
        assert abs(float(got[0::op.b].mean())) < 1e-13


@pytest.mark.parametrize("gamma", [0, 1])
def test_project_kernel_noalloc_stokes_one_call_per_field(lib, gamma):
    """A Stokes vector (fields u_1..u_dim, p per element) is projected with one
    call per field at offset f * field_b and stride b, and then equals the
    allocating call, which removes every field's constant."""
    gen = torch.Generator(device="cuda").manual_seed(5)
    op = lib.Operator(2, 12, 2, stokes=gamma)
    assert op.nfields == 3
    v = torch.randn(op.size, dtype=torch.float64, device="cuda", generator=gen)
    ref = op.project_kernel(v.clone())
    got = v.clone()
    for f in range(op.nfields):
        lib.project_kernel_noalloc(got, op.N, op.b, offset=f * op.field_b)
    torch.cuda.synchronize()
    assert float((got - ref).abs().max() / ref.abs().max()) < 1e-14
    # one call alone is the scalar contract: it leaves the other fields' constants
    one = lib.project_kernel_noalloc(v.clone(), op.N, op.b)
    torch.cuda.synchronize()
    assert float((one - ref).abs().max()) > 1e-6


@pytest.mark.parametrize("N", [16777216, 4096 * 3 + 1, 4096, 1])
def test_project_kernel_noalloc_sizes(lib, N):
    """N = the maximum fills every partial-sum slot of the fixed scratch; 4096k + 1
    has a last chunk of one element.  b = 1: the whole vector is the mode-0 data."""
    assert lib.NOALLOC_MAX_ELEMENTS == 16777216
    gen = torch.Generator(device="cuda").manual_seed(N % 1000)
    v = torch.rand(N, dtype=torch.float64, device="cuda", generator=gen) + 3.0
    ref = v - v.mean()
    got = lib.project_kernel_noalloc(v.clone(), N, 1)
    torch.cuda.synchronize()
    assert float((got - ref).abs().max()) < 1e-12
    assert abs(float(got.mean())) < 1e-12


def test_project_kernel_noalloc_rejects_bad_input(lib):
    v = torch.zeros(8, dtype=torch.float64, device="cuda")
    # the C entry point refuses the size itself (before touching v)
    st = lib._lib.ldgmg_project_kernel_noalloc(lib.NOALLOC_MAX_ELEMENTS + 1, 1, lib._ptr(v), None)
    assert st == lib.EINVAL and "exceeds the maximum" in lib._lib.ldgmg_last_error().decode()
    with pytest.raises(lib.LdgmgError) as e:
        lib.project_kernel_noalloc(v, lib.NOALLOC_MAX_ELEMENTS + 1, 1)
    assert e.value.status == lib.EINVAL and "exceeds the maximum" in str(e.value)
    # the wrapper refuses what the C call cannot check: a vector too short for N and b
    with pytest.raises(lib.LdgmgError) as e:
        lib.project_kernel_noalloc(v, 3, 4)
    assert e.value.status == lib.EINVAL
    with pytest.raises(lib.LdgmgError):
        lib.project_kernel_noalloc(v.float(), 8, 1)
