"""Failure detection without a GPU fault: a device wait that nothing satisfies gives up after
its bound, the library reports FP_ETIMEOUT, and the context keeps working."""
import numpy as np
import pytest

import workloads
from oracle import field
from tests._gpu import to_dev, torch_dev

pytestmark = pytest.mark.gpu


def test_bounded_wait_times_out_and_context_survives():
    torch, dev = torch_dev()
    import __graft_entry__ as g
    g.build()
    import paper_0809_0063_gb300 as fp
    ctx = fp.fp_ctx_create(0)
    try:
        fp.fp_selftest_bounded_wait(ctx, 1000)
        with pytest.raises(fp.FpError) as ei:
            fp.fp_ctx_status(ctx)
        assert ei.value.status == fp.FP_ETIMEOUT
        fp.fp_ctx_status(ctx)            # flag cleared
        a, b = workloads.matmul_inputs(9, 3, 64, 64, 64)
        C = torch.empty((64, 64), dtype=torch.uint8, device=dev)
        fp.fp_matmul(ctx, 3, 64, 64, 64, to_dev(torch, dev, a), 64, to_dev(torch, dev, b), 64, C, 64,
                     fp.FP_MM_PLAIN_TC)
        fp.fp_ctx_status(ctx)
        assert np.array_equal(C.cpu().numpy(), field.matmul_mod(a, b, 3))
    finally:
        fp.fp_ctx_destroy(ctx)
