"""poly_estimate_batched (one captured CUDA graph per batch) and the contraction autotuner.

A batch mixes grid sizes and precisions, several fields per plan; its results
must equal the single-field calls bit for bit, on the first (captured) call and
on replays, also after the fields' contents change in place.  Tuning may only
reorder the final FP64 sums: the tuned plan agrees with the untuned one within
the split-BF16 bound, repeats itself bit for bit, and a configuration code
restored on a fresh plan (directly or through the JSON cache) reproduces it.
"""
import numpy as np
import pytest

import fieldgen

torch = pytest.importorskip("torch")
import paper_1904_11055_gb300 as ps  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1904_11055_gb300 import build

    build.build()


def _field(kind, N, seed):
    return torch.from_numpy(fieldgen.field(kind, N, seed, np.float32)).cuda()


def test_graph_batch_of_mixed_sizes_matches_single_calls():
    specs = [(32, 8, "fp32"), (48, 12, "split_bf16"), (24, 7, "fp32")]
    plans = [ps.Plan(N, 500.0, 3, fieldgen.unit_edges(ns), prec) for N, ns, prec in specs]
    bplans, fields = [], []
    for r in range(3):  # three fields per plan, interleaved
        for j, (N, _, _) in enumerate(specs):
            bplans.append(plans[j])
            fields.append(_field("lognormal", N, 100 + 10 * r + j))
    outs = [torch.full((p.nbins,), float("nan"), dtype=torch.float64, device="cuda") for p in bplans]

    def singles():
        return [p.estimate(f).cpu().numpy() for p, f in zip(bplans, fields)]

    ref = singles()
    for _ in range(2):  # capture, then replay
        ps.estimate_batched(bplans, fields, outs)
        torch.cuda.synchronize()
        for o, s in zip(outs, ref):
            assert np.array_equal(o.cpu().numpy(), s)
    # the graph reads the fields where they live: new contents, same addresses
    for k, f in enumerate(fields):
        f.copy_(_field("gaussian", f.shape[0], 200 + k))
    ref2 = singles()
    ps.estimate_batched(bplans, fields, outs)
    torch.cuda.synchronize()
    for o, s, s_old in zip(outs, ref2, ref):
        assert np.array_equal(o.cpu().numpy(), s)
        assert not np.array_equal(s, s_old)


def test_destroying_a_plan_drops_its_graphs():
    a = ps.Plan(32, 500.0, 3, fieldgen.unit_edges(8), "fp32")
    b = ps.Plan(24, 500.0, 3, fieldgen.unit_edges(7), "fp32")
    fa, fb = _field("lognormal", 32, 1), _field("lognormal", 24, 2)
    outs = ps.estimate_batched([a, b], [fa, fb])
    torch.cuda.synchronize()
    b.close()
    out_a = ps.estimate_batched([a], [fa])[0]
    torch.cuda.synchronize()
    assert np.array_equal(out_a.cpu().numpy(), outs[0].cpu().numpy())


def test_tuning_reorders_only_the_final_sums(tmp_path):
    N, L, e = 64, 1000.0, fieldgen.unit_edges(16)
    d = _field("lognormal", N, 7)
    plan = ps.Plan(N, L, 3, e, "split_bf16")
    B0, scale = plan.estimate(d, scale=True)
    cfg, ms = plan.tune(d)
    assert cfg != 0 and ms > 0
    B1 = plan.estimate(d)
    B2 = plan.estimate(d)
    assert torch.equal(B1, B2)
    c_n = (L ** 3) ** 2 / float(N ** 3) ** 3
    assert ((B1 - B0).abs() / (c_n * scale)).max().item() <= 1e-5
    fresh = ps.Plan(N, L, 3, e, "split_bf16")
    fresh.set_config(cfg)
    assert torch.equal(fresh.estimate(d), B1)
    # the JSON cache: the first call tunes and records, a later plan restores without timing
    cache = str(tmp_path / "tune.json")
    c1 = ps.autotune(ps.Plan(N, L, 3, e, "split_bf16"), d, cache)
    p2 = ps.Plan(N, L, 3, e, "split_bf16")
    assert ps.autotune(p2, d, cache) == c1
    p3 = ps.Plan(N, L, 3, e, "split_bf16")
    p3.set_config(c1)
    assert torch.equal(p2.estimate(d), p3.estimate(d))


def test_tuning_has_nothing_to_do_for_cuda_core_plans():
    plan = ps.Plan(32, 500.0, 3, fieldgen.unit_edges(8), "fp32")
    assert plan.tune(_field("lognormal", 32, 3)) == (0, 0.0)


@pytest.mark.parametrize("prec", ["fp32", "split_bf16", "fp64"])
def test_closing_a_plan_leaves_no_pending_cuda_error(prec):
    """Teardown frees every buffer once: a stale error would surface at the next kernel launch anywhere."""
    N, e = 32, fieldgen.unit_edges(8)
    plan = ps.Plan(N, 500.0, 3, e, prec)
    dt = torch.float64 if prec == "fp64" else torch.float32
    d = _field("lognormal", N, 11).to(dt)
    plan.estimate(d)
    plan.backward(d, torch.ones(plan.nbins, dtype=torch.float64, device="cuda"))
    torch.cuda.synchronize()
    plan.close()
    assert (torch.ones(8, device="cuda") * 2).sum().item() == 16.0
