"""GPU test of mz_zeta_noalloc, the zeta entry point that allocates nothing.

Some callers cannot allocate device memory when they call the transform (for
example code running inside another allocator's callbacks, or a loop that must
not block on the driver's allocator). For them the library keeps a fixed
scratch array and mz_zeta_noalloc uses it instead of a caller workspace. This
file checks, through the C ABI, that two calls in a row give the same results
as mz_zeta with a workspace, and that a transform too large for the array is
refused. It is named so that pytest collects it after every other test file.
"""
import numpy as np
import pytest
import torch

import posetgen as pg
import paper_2211_13706_gb300 as mz
from gpu_util import TOL

pytestmark = pytest.mark.gpu


def _device_values(n, batch, dtype, seed):
    if dtype == mz.MZ_I64:
        x = pg.function_values(n, batch, "i64:1000", seed)
        return torch.from_numpy(x).cuda()
    if dtype == mz.MZ_F64:
        return torch.from_numpy(pg.function_values(n, batch, "f64u", seed)).cuda()
    hi = pg.function_values(n, batch, "f32u", seed)
    return torch.from_numpy(np.stack([hi, np.zeros_like(hi)])).cuda()


def _close(a, b, dtype):
    if dtype == mz.MZ_I64:
        return torch.equal(a, b)
    a64, b64 = a.double(), b.double()
    if dtype == mz.MZ_F32C:
        a64, b64 = a64[0] + a64[1], b64[0] + b64[1]
    scale = b64.abs().max().item() or 1.0
    return (a64 - b64).abs().max().item() <= TOL[dtype] * scale


@pytest.mark.parametrize("dtype", [mz.MZ_I64, mz.MZ_F64, mz.MZ_F32C])
def test_noalloc_matches_workspace_path_twice(dtype):
    p = pg.planted_chain_poset(4096, 16, 1, cross_p=4 / 4096)
    plan = mz.Plan(p.n, p.src, p.dst, p.chain_id)
    stream = torch.cuda.current_stream().cuda_stream
    ws, wsb = plan.workspace(dtype, 1)
    for call, seed in enumerate((1, 2)):          # two calls in a row, different inputs
        f = _device_values(p.n, 1, dtype, seed)
        if dtype != mz.MZ_F32C:
            f = f[:, 0].contiguous()
        want = torch.empty_like(f)
        got = torch.full_like(f, 7)
        mz.mz_zeta(plan.handle, dtype, f.data_ptr(), want.data_ptr(), 1, ws, wsb, stream)
        mz.mz_zeta_noalloc(plan.handle, dtype, f.data_ptr(), got.data_ptr(), 1, stream)
        mz.mz_check(plan.handle, stream)
        assert _close(got, want, dtype), f"call {call}"


def test_noalloc_batched_and_size_limit():
    p = pg.planted_chain_poset(4096, 16, 2, cross_p=4 / 4096)
    plan = mz.Plan(p.n, p.src, p.dst, p.chain_id)
    stream = torch.cuda.current_stream().cuda_stream
    f = _device_values(p.n, 8, mz.MZ_I64, 3)
    want = plan.zeta(f)
    got = torch.empty_like(f)
    mz.mz_zeta_noalloc(plan.handle, mz.MZ_I64, f.data_ptr(), got.data_ptr(), 8, stream)
    mz.mz_check(plan.handle, stream)
    assert torch.equal(got, want)
    # (n + k) * batch * 8 bytes of prefixes alone exceed the 16 MiB array: refused, nothing launched
    big = 1024
    assert mz.mz_workspace_size(plan.handle, mz.MZ_I64, big) > mz.MZ_NOALLOC_SCRATCH_BYTES
    x = torch.zeros(p.n, big, dtype=torch.int64, device="cuda")
    y = torch.zeros_like(x)
    with pytest.raises(mz.MzError) as e:
        mz.mz_zeta_noalloc(plan.handle, mz.MZ_I64, x.data_ptr(), y.data_ptr(), big, stream)
    assert e.value.status == mz.MZ_ERR_INVALID_ARG
    assert "scratch" in str(e.value)


def test_noalloc_at_the_size_limit():
    """The largest batch whose workspace (mz_workspace_size) fits the fixed array runs and
    matches mz_zeta exactly; one more column does not fit and is refused."""
    p = pg.planted_chain_poset(4096, 16, 4, cross_p=4 / 4096)
    plan = mz.Plan(p.n, p.src, p.dst, p.chain_id)
    limit = mz.MZ_NOALLOC_SCRATCH_BYTES
    fits = [b for b in range(1, 4096) if mz.mz_workspace_size(plan.handle, mz.MZ_I64, b) <= limit]
    bmax = max(fits)
    assert mz.mz_workspace_size(plan.handle, mz.MZ_I64, bmax + 1) > limit
    stream = torch.cuda.current_stream().cuda_stream
    for b, ok in ((bmax, True), (bmax + 1, False)):
        f = _device_values(p.n, b, mz.MZ_I64, 5)
        got = torch.empty_like(f)
        if ok:
            mz.mz_zeta_noalloc(plan.handle, mz.MZ_I64, f.data_ptr(), got.data_ptr(), b, stream)
            mz.mz_check(plan.handle, stream)
            assert torch.equal(got, plan.zeta(f))
        else:
            with pytest.raises(mz.MzError) as e:
                mz.mz_zeta_noalloc(plan.handle, mz.MZ_I64, f.data_ptr(), got.data_ptr(), b, stream)
            assert e.value.status == mz.MZ_ERR_INVALID_ARG
