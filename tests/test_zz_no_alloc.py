"""cs_lambda_max_noalloc: the allocation-free Lipschitz estimate.

It serves callers that cannot allocate device memory (a process whose HBM was
reserved in full at start-up, or a loop that cannot take cudaMalloc's implicit
device synchronisation).  Checked through the C ABI against the plan's L from
cs_make_phi (which allocates its own scratch), on two calls in a row that
share the built-in scratch array.  This file is collected last on purpose.
"""
import gc

import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1311_1419_gb300 import binding
    return binding


def test_noalloc_lambda_matches_make_phi_on_two_calls_in_a_row(B):
    ctx = B.cs_ctx_create(0)
    plans = []
    try:
        # the second call is smaller than the first: stale scratch from the
        # first call must not leak into it; the third repeats the first
        cases = [(256, 128, 0), (1024, 102, 3), (256, 128, 0)]
        out = torch.full((len(cases),), float("nan"), dtype=torch.float64, device="cuda")
        stream = torch.cuda.current_stream()
        for i, (n, m, seed) in enumerate(cases):
            plan = B.cs_make_phi(ctx, n, m, seed)
            plans.append(plan)
            B.cs_lambda_max_noalloc(B.cs_plan_phi(plan), n, m, out[i:i + 1], stream)
        torch.cuda.synchronize()
        got = out.cpu().tolist()
        for (n, m, seed), lam, plan in zip(cases, got, plans):
            assert 1.0001 * lam == pytest.approx(B.cs_plan_lipschitz(plan), rel=1e-10)
        assert got[0] == got[2]
    finally:
        for p in plans:
            B.cs_plan_destroy(p)
        B.cs_ctx_destroy(ctx)


def test_noalloc_rejects_sizes_beyond_its_scratch(B):
    phi = torch.zeros((257, 300), dtype=torch.float32, device="cuda")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(B.CsError) as ei:
        B.cs_lambda_max_noalloc(phi, 300, 257, out)
    assert ei.value.status == B.CS_EINVAL
    assert "256" in B.cs_last_error()


def test_noalloc_calls_leave_device_memory_unchanged(B):
    """After a first call (which looks up the array's address), further calls
    change neither the device's free memory nor torch's allocations: nothing
    is allocated and kept."""
    ctx = B.cs_ctx_create(0)
    plan = B.cs_make_phi(ctx, 256, 96, 5)
    try:
        out = torch.zeros(1, dtype=torch.float64, device="cuda")
        phi = B.cs_plan_phi(plan)
        B.cs_lambda_max_noalloc(phi, 256, 96, out)
        torch.cuda.synchronize()
        # tensors earlier tests left for the garbage collector must not be freed
        # inside the measured window
        gc.collect()
        gc.disable()
        try:
            free0, _ = torch.cuda.mem_get_info()
            alloc0 = torch.cuda.memory_allocated()
            for _ in range(3):
                B.cs_lambda_max_noalloc(phi, 256, 96, out)
            torch.cuda.synchronize()
            free1, _ = torch.cuda.mem_get_info()
            alloc1 = torch.cuda.memory_allocated()
        finally:
            gc.enable()
        assert free1 == free0
        assert alloc1 == alloc0
        assert 1.0001 * out.item() == pytest.approx(B.cs_plan_lipschitz(plan), rel=1e-10)
    finally:
        B.cs_plan_destroy(plan)
        B.cs_ctx_destroy(ctx)
