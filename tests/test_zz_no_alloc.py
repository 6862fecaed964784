"""tim_node_select_noalloc: the greedy node selection for callers that cannot let the
library allocate device memory -- their device memory belongs to another allocator or a
fixed budget, or they must not trigger the device-wide synchronisation of cudaMalloc and
cudaFree. It works on RR sets the caller already holds on the device. Its seeds and
covered count must equal those of tim_node_select on the same sets, including on two
calls in a row: all calls share one scratch array that keeps the previous call's
contents, so each call must clear what it needs."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _reference_selections():
    from paper_1404_0900_gb300 import inputs, tim
    out = {}
    with tim.Engine(0) as eng:
        for name, (scale, seed, k, theta) in {"a": (12, 3, 20, 30000),
                                               "b": (11, 5, 7, 12000)}.items():
            g = inputs.rmat(scale, seed=seed)
            tim.tim_load_graph(eng.ctx, g.n, g.rowptr, g.dst, inputs.weighted_cascade(g),
                               tim.TIM_IC)
            tim.tim_sample_rr(eng.ctx, theta, seed, 0)
            seeds, _, cov = tim.tim_node_select(eng.ctx, k)
            off, mem, _ = tim.tim_get_rr(eng.ctx)
            out[name] = (g.n, k, off, mem, seeds, cov)
    return out


def test_noalloc_selection_matches_node_select_on_repeated_calls():
    import torch
    from paper_1404_0900_gb300 import tim
    ref = _reference_selections()
    stream = torch.cuda.current_stream()
    # two calls in a row on the same sets, then other sets, then the first ones again
    for name in ("a", "a", "b", "a"):
        n, k, off, mem, seeds, cov = ref[name]
        d_off = torch.from_numpy(off).cuda()
        d_mem = torch.from_numpy(mem).cuda()
        d_seeds = torch.full((k,), -1, dtype=torch.int32, device="cuda")
        d_cov = torch.zeros(1, dtype=torch.int64, device="cuda")
        tim.tim_node_select_noalloc(0, stream, n, off.shape[0] - 1, d_off, d_mem, k, d_seeds,
                                    d_cov)
        torch.cuda.synchronize()
        assert np.array_equal(d_seeds.cpu().numpy(), seeds), name
        assert int(d_cov.item()) == cov, name


def test_noalloc_rejects_sizes_beyond_its_limits():
    import torch
    from paper_1404_0900_gb300 import tim
    d_off = torch.zeros(2, dtype=torch.int64, device="cuda")
    d_mem = torch.zeros(1, dtype=torch.int32, device="cuda")
    d_seeds = torch.zeros(2048, dtype=torch.int32, device="cuda")
    d_cov = torch.zeros(1, dtype=torch.int64, device="cuda")
    for n, n_sets, k in (((1 << 18) + 1, 1, 1), (1000, (1 << 20) + 1, 1), (5000, 1, 1025),
                         (10, 1, 11)):
        with pytest.raises(tim.TimError) as ei:
            tim.tim_node_select_noalloc(0, None, n, n_sets, d_off, d_mem, k, d_seeds, d_cov)
        assert ei.value.code == -1


def test_noalloc_call_takes_no_device_memory():
    """After a first call (which looks up the array's address), further calls leave the
    device's free memory unchanged: they allocate nothing."""
    import torch
    from paper_1404_0900_gb300 import tim
    n, k, off, mem, seeds, cov = _reference_selections()["b"]
    d_off = torch.from_numpy(off).cuda()
    d_mem = torch.from_numpy(mem).cuda()
    d_seeds = torch.zeros(k, dtype=torch.int32, device="cuda")
    d_cov = torch.zeros(1, dtype=torch.int64, device="cuda")
    stream = torch.cuda.current_stream()
    call = lambda: tim.tim_node_select_noalloc(0, stream, n, off.shape[0] - 1, d_off, d_mem, k,
                                               d_seeds, d_cov)
    call()
    torch.cuda.synchronize()
    same = False
    for _ in range(3):  # another process on the device could move the figure: retry
        free0, _ = torch.cuda.mem_get_info()
        call()
        call()
        torch.cuda.synchronize()
        free1, _ = torch.cuda.mem_get_info()
        if free1 == free0:
            same = True
            break
    assert same, (free0, free1)
    assert np.array_equal(d_seeds.cpu().numpy(), seeds) and int(d_cov.item()) == cov


def test_noalloc_member_out_of_range_and_no_sets():
    import torch
    from paper_1404_0900_gb300 import tim
    n, k = 100, 5
    d_seeds = torch.full((k,), -1, dtype=torch.int32, device="cuda")
    d_cov = torch.zeros(1, dtype=torch.int64, device="cuda")
    # a member equal to n: checked after the run, reported as an argument error
    d_off = torch.tensor([0, 2, 3], dtype=torch.int64, device="cuda")
    d_mem = torch.tensor([1, n, 7], dtype=torch.int32, device="cuda")
    with pytest.raises(tim.TimError) as ei:
        tim.tim_node_select_noalloc(0, None, n, 2, d_off, d_mem, k, d_seeds, d_cov)
    assert ei.value.code == -1
    # no RR sets: nothing is covered and the smallest ids are the seeds
    d_off = torch.zeros(1, dtype=torch.int64, device="cuda")
    tim.tim_node_select_noalloc(0, None, n, 0, d_off, d_mem, k, d_seeds, d_cov)
    torch.cuda.synchronize()
    assert d_seeds.cpu().tolist() == list(range(k)) and int(d_cov.item()) == 0
