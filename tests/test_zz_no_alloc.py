"""The allocation-free evaluation entry point, through the C ABI.

ebic_eval_population_noalloc serves callers that cannot let a library allocate GPU memory: a
framework that has already reserved the device memory in its own pool, or a latency-critical
loop that cannot afford cudaMalloc/cudaFree.  Its results must equal those of the regular entry
point, ebic_eval_population, exactly (the counts are integers), on two calls in a row: the second
call reuses the static scratch array the first one left behind.  This file is collected last, so
that a run stopping at the first failure has already run every other test."""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ebic():
    from paper_2105_01196_gb300 import ebic as e
    return e


def make_inputs(seed, R, C, n):
    g = np.random.default_rng(seed)
    x = (g.integers(-3, 4, size=(R, C)) * 0.5).astype(np.float32)   # many ties
    x[g.random((R, C)) < 0.03] = -0.0
    lens = g.integers(2, min(64, C) + 1, size=n)
    off = np.zeros(n + 1, np.int32)
    off[1:] = np.cumsum(lens)
    ci = np.concatenate([g.choice(C, size=int(L), replace=False) for L in lens]).astype(np.int32)
    return x, ci, off


def test_noalloc_matches_regular_entry_point_twice(ebic):
    torch = pytest.importorskip("torch")
    dev = torch.device("cuda:0")
    stream = torch.cuda.current_stream()
    cases = [make_inputs(1, 3001, 40, 700), make_inputs(2, 130, 70, 3000)]
    for neg, num, den, ns, lk in ((1, 85, 100, 0, 0), (0, 1, 1, 0, 0), (1, 85, 100, 1, 1),
                                  (1, 2, 3, 1, 0), (0, 2, 3, 0, 1)):
        p = ebic.Params.make(neg_trends=neg, ratio_num=num, ratio_den=den, mode=ebic.MODE_DIRECT,
                             non_strict=ns, last_kept=lk)
        for x, ci, off in cases:
            n = len(off) - 1
            with ebic.Context(0) as ctx:
                ctx.load_matrix(x)
                want = ctx.eval_population(ci, off, p)
            x_cm = torch.from_numpy(np.ascontiguousarray(x.T)).to(dev)
            ci_d = torch.from_numpy(ci).to(dev)
            off_d = torch.from_numpy(off).to(dev)
            for _call in range(2):
                outs = [torch.full((n,), -7, dtype=torch.int32, device=dev) for _ in range(3)]
                outs.append(torch.full((n,), -7, dtype=torch.int64, device=dev))
                ebic.ebic_eval_population_noalloc(x_cm, ci_d, off_d, p, *outs, device=0,
                                                  stream=stream.cuda_stream)
                got = [o.cpu().numpy() for o in outs]
                for g_, w_ in zip(got, want):
                    assert np.array_equal(np.asarray(g_, np.int64), np.asarray(w_, np.int64))


def test_noalloc_rejects_what_it_cannot_do(ebic):
    torch = pytest.importorskip("torch")
    dev = torch.device("cuda:0")
    p = ebic.Params.make()
    x = torch.zeros((4, 10), dtype=torch.float32, device=dev)      # 4 columns x 10 rows
    big = ebic.NOALLOC_MAX_IND + 1
    off = torch.arange(0, 2 * (big + 1), 2, dtype=torch.int32, device=dev)
    ci = torch.tensor([0, 1] * big, dtype=torch.int32, device=dev)
    with pytest.raises(ebic.EbicError) as e:
        ebic.ebic_eval_population_noalloc(x, ci, off, p)
    assert e.value.code == ebic.EBIC_EINVAL and "EBIC_NOALLOC_MAX_IND" in str(e.value)
    ci_h = np.array([0, 1], np.int32)
    off_h = np.array([0, 2], np.int32)
    with pytest.raises(ebic.EbicError) as e:
        ebic.ebic_eval_population_noalloc(x, ci_h, off_h, p)       # host population
    assert e.value.code == ebic.EBIC_EINVAL
    xn = x.clone()
    xn[2, 3] = float("nan")
    with pytest.raises(ebic.EbicError) as e:
        ebic.ebic_eval_population_noalloc(xn, ci[:2].contiguous(), off[:2].contiguous(), p)
    assert e.value.code == ebic.EBIC_ENAN
