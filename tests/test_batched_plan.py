"""The batched launch's task order, checked on the host (no GPU).

The persistent task-graph kernel takes tasks in the order of one merged list
and every task waits only for flags raised by other tasks; it cannot
deadlock when every dependency sits earlier in that list.  The library
rebuilds the list with the same decoding and merge formulas as the device
plan and counts dependencies that are not earlier, and list slots that do not
hold exactly one task; both must be zero for any batch, in both forms and
for any tile threshold of the mixed form.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.filterwarnings("ignore")


@pytest.fixture(scope="module")
def g():
    from paper_1305_4886_gb300 import build, gp
    build.build()
    return gp


def _ns(seed, k, lo, hi):
    rng = np.random.default_rng(seed)
    return np.rint(np.exp(rng.uniform(np.log(lo), np.log(hi), size=k))).astype(np.int64).tolist()


@pytest.mark.parametrize("precision", ["fp64", "mixed_f16"])
@pytest.mark.parametrize("ns", [
    [1], [64], [65], [128], [129], [1, 1, 1], [4096],
    [3, 700, 64, 1300, 129, 511, 512, 513],
])
def test_small_batches_have_a_topological_order(g, precision, ns):
    nt, bad_order, bad_slots = g.gp_batched_plan_check(ns, precision)
    assert nt > 0 and bad_order == 0 and bad_slots == 0


@pytest.mark.parametrize("threshold", [0, 256, 700, 1 << 20])
def test_config5_sizes_with_every_tile_threshold(g, threshold):
    ns = _ns(48865, 512, 256, 4096)
    nt, bad_order, bad_slots = g.gp_batched_plan_check(ns, "mixed_f16", threshold)
    assert nt > 0 and bad_order == 0 and bad_slots == 0


def test_fp64_config5_sizes(g):
    nt, bad_order, bad_slots = g.gp_batched_plan_check(_ns(48865, 512, 256, 4096), "fp64")
    assert bad_order == 0 and bad_slots == 0
    # the FP64 form's list: T(T+1)/2 Cholesky + solve + T(T-1)/2 inverse + T(T+1)/2 gradient + final
    T = [(n + 63) // 64 for n in _ns(48865, 512, 256, 4096)]
    assert nt == sum(t * (t + 1) // 2 + 1 + t * (t - 1) // 2 + t * (t + 1) // 2 + 1 for t in T)


def test_many_problems_and_one_large(g):
    ns = [1 + (7 * i) % 300 for i in range(2000)] + [20000]
    nt, bad_order, bad_slots = g.gp_batched_plan_check(ns, "mixed_f16", 200)
    assert bad_order == 0 and bad_slots == 0


def test_invalid_arguments(g):
    from paper_1305_4886_gb300.gp import GpError
    with pytest.raises(GpError):
        g.gp_batched_plan_check([0], "mixed_f16")
    with pytest.raises(GpError):
        g.gp_batched_plan_check([10], "emu_fp64")
