"""Failure detection without a GPU fault: every device-side wait of the search
kernel (team barriers, the k-list lock) has a clock64 budget.  With a budget of
one cycle the first wait runs out; the kernel records TKC_ETIMEOUT, every block
returns, the call reports the error, and the context stays usable: the next
call with the default budget returns the exact top-k."""
import numpy as np
import pytest

import oracle
from paper_1704_01077_gb300 import graphgen as gg

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("order_name,teams", [("deg", 2), ("nb", 0)])
def test_wait_budget_runs_out_and_context_recovers(gpu_lib, order_name, teams):
    t = gpu_lib
    order = t.TKC_ORDER_NB if order_name == "nb" else t.TKC_ORDER_DEG
    g = gg.rmat(13, 16, seed=21)
    ref = oracle.textbook_topk(g, 10, threads=0)
    ctx = t.tkc_create(t.Options(order=order, batch_bits=64, teams=teams, timeout_cycles=1))
    try:
        h = t.tkc_load_csr(ctx, g.n, g.offsets, g.cols, g.directed)
        try:
            with pytest.raises(t.TkcError) as err:
                t.tkc_topk_closeness(h, 10)
            assert err.value.code == t.TKC_ETIMEOUT
            t.tkc_set_options(ctx, t.Options(order=order, batch_bits=64, teams=teams))
            for _ in range(2):
                res = t.tkc_topk_closeness(h, 10)
                assert list(res.ids) == list(ref.ids)
                assert np.array_equal(res.dist_sum, ref.S) and np.array_equal(res.reach, ref.r)
                assert res.n_tied_at_kth == ref.n_tied
        finally:
            t.tkc_free_graph(h)
    finally:
        t.tkc_destroy(ctx)
