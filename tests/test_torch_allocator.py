"""Plan memory through PyTorch's caching allocator (mz_build_opts::dev_alloc / dev_free,
Python `torch_allocator=True`): the plan's buffers are counted by
torch.cuda.memory_allocated, given back on close, and the transforms are unchanged."""
import pytest

import posetgen as pg
import paper_2211_13706_gb300 as mz

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("device_build", [False, True])
def test_plan_memory_through_torch(device_build):
    import torch
    p = pg.planted_chain_poset(20000, 24, 3, cross_deg=2)
    torch.cuda.synchronize()
    base = torch.cuda.memory_allocated()
    plan = mz.Plan(p.n, p.src, p.dst, p.chain_id, build_transpose=True, torch_allocator=True,
                   device_build=device_build)
    torch.cuda.synchronize()
    held = torch.cuda.memory_allocated() - base
    assert held >= plan.info["device_bytes"] > 0
    ref = mz.Plan(p.n, p.src, p.dst, p.chain_id, build_transpose=True)
    x = torch.from_numpy(pg.function_values(p.n, 2, "i64:1000", 3)).cuda()
    for op in ("zeta", "mobius", "zeta_T", "mobius_T"):
        a, b = getattr(plan, op)(x), getattr(ref, op)(x)
        plan.check()
        assert torch.equal(a, b), op
    torch.cuda.synchronize()
    before_close = torch.cuda.memory_allocated()
    bytes_ = plan.info["device_bytes"]
    plan.close()
    torch.cuda.synchronize()
    assert before_close - torch.cuda.memory_allocated() >= bytes_
    ref.close()
