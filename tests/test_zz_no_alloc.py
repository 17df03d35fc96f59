"""The allocation-free evaluation entry point, through the C ABI.

ebic_eval_population_noalloc serves callers that cannot let a library allocate GPU memory: a
framework that has already reserved the device memory in its own pool, or a latency-critical
loop that cannot afford cudaMalloc/cudaFree.  Its results must equal those of the regular entry
point, ebic_eval_population, and those of the CPU oracle exactly (the counts are integers), on
two calls in a row: the second call reuses the static scratch array the first one left behind.
This file is collected last, so that a run stopping at the first failure has already run every
other test."""

import ctypes

import numpy as np
import pytest

from oracle import counts as ocounts
from oracle.params import Params as OParams

pytestmark = pytest.mark.gpu

VARIANTS = ((1, 85, 100, 0, 0), (0, 1, 1, 0, 0), (1, 85, 100, 1, 1), (1, 2, 3, 1, 0),
            (0, 2, 3, 0, 1))


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


def make_subnormal_inputs(seed, R, C, n):
    """Values drawn from a small set that holds ties, both signed zeros and subnormals of both
    signs next to each other (the cases a flush-to-zero or a sign mistake would change)."""
    g = np.random.default_rng(seed)
    tiny = np.float32(1e-45)                             # smallest positive subnormal
    vals = np.array([-1.0, -np.float32(1e-40), -tiny, -0.0, 0.0, tiny, np.float32(2e-45),
                     np.float32(1e-40), np.float32(1.2e-38), 0.5, 1.0], dtype=np.float32)
    x = vals[g.integers(0, len(vals), size=(R, C))]
    lens = g.integers(2, min(64, C) + 1, size=n)
    off = np.zeros(n + 1, np.int32)
    off[1:] = np.cumsum(lens)
    ci = np.concatenate([g.choice(C, size=int(L), replace=False) for L in lens]).astype(np.int32)
    return x, ci, off


def _outs(torch, n, dev):
    outs = [torch.full((n,), -7, dtype=torch.int32, device=dev) for _ in range(3)]
    outs.append(torch.full((n,), -7, dtype=torch.int64, device=dev))
    return outs


def _same(got, want):
    return all(np.array_equal(np.asarray(g_, np.int64), np.asarray(w_, np.int64))
               for g_, w_ in zip(got, want))


def test_noalloc_matches_regular_entry_point_twice(ebic):
    torch = pytest.importorskip("torch")
    dev = torch.device("cuda:0")
    stream = torch.cuda.current_stream()
    cases = [make_inputs(1, 3001, 40, 700), make_inputs(2, 130, 70, 3000)]
    for neg, num, den, ns, lk in VARIANTS:
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
                outs = _outs(torch, n, dev)
                ebic.ebic_eval_population_noalloc(x_cm, ci_d, off_d, p, *outs, device=0,
                                                  stream=stream.cuda_stream)
                assert _same([o.cpu().numpy() for o in outs], want)


def test_noalloc_matches_oracle_on_subnormals_signed_zeros_and_ties(ebic):
    """Element-wise equality with the CPU oracle's plain definition (strict float32 comparisons,
    -0 equal to +0, subnormals kept), in every pair-test variant, on two calls in a row."""
    torch = pytest.importorskip("torch")
    dev = torch.device("cuda:0")
    stream = torch.cuda.current_stream()
    x, ci, off = make_subnormal_inputs(5, 1037, 67, 400)
    n = len(off) - 1
    x_cm = torch.from_numpy(np.ascontiguousarray(x.T)).to(dev)
    ci_d, off_d = torch.from_numpy(ci).to(dev), torch.from_numpy(off).to(dev)
    for neg, num, den, ns, lk in VARIANTS:
        p = ebic.Params.make(neg_trends=neg, ratio_num=num, ratio_den=den, non_strict=ns,
                             last_kept=lk)
        op = OParams(neg_trends=neg, ratio_num=num, ratio_den=den, min_rows=p.min_rows,
                     col_cap=p.col_cap, non_strict=ns, last_kept=lk)
        want = ocounts.eval_population(x, ci, off, op)
        for _call in range(2):
            outs = _outs(torch, n, dev)
            ebic.ebic_eval_population_noalloc(x_cm, ci_d, off_d, p, *outs, device=0,
                                              stream=stream.cuda_stream)
            assert _same([o.cpu().numpy() for o in outs], want), (neg, num, den, ns, lk)


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
    # host memory, through the C ABI directly (the binding rejects it before the call)
    ci_h = np.array([0, 1], np.int32)
    off_h = np.array([0, 2], np.int32)
    buf = ctypes.create_string_buffer(256)
    st = ebic.lib().ebic_eval_population_noalloc(
        ebic.ptr(x), 10, 4, ebic.ptr(ci_h), ebic.ptr(off_h), 1, ctypes.byref(p), None, None,
        None, None, 0, None, buf, 256)
    assert st == ebic.EBIC_EINVAL and b"device memory" in buf.value
    with pytest.raises(ebic.EbicError) as e:
        ebic.ebic_eval_population_noalloc(x, ci_h, off_h, p)
    assert e.value.code == ebic.EBIC_EINVAL
    xn = x.clone()
    xn[2, 3] = float("nan")
    with pytest.raises(ebic.EbicError) as e:
        ebic.ebic_eval_population_noalloc(xn, ci[:2].contiguous(), off[:2].contiguous(), p)
    assert e.value.code == ebic.EBIC_ENAN


def test_noalloc_rejects_bad_chromosomes_on_the_device(ebic):
    """The device-side chromosome check is the only guard before the kernel indexes the matrix
    with caller column ids: a repeated column, a column out of range (either side) and a length
    outside [2, 64] are each rejected, and a valid call on the same device afterwards is still
    correct."""
    torch = pytest.importorskip("torch")
    dev = torch.device("cuda:0")
    p = ebic.Params.make(neg_trends=1, ratio_num=85, ratio_den=100)
    x, ci_ok, off_ok = make_inputs(9, 300, 70, 50)
    x_cm = torch.from_numpy(np.ascontiguousarray(x.T)).to(dev)
    bad_cases = [
        [[0, 1, 2], [3, 4, 3]],                 # repeated column
        [[0, 1], [5, 70]],                      # column == cols
        [[0, 1], [-1, 2]],                      # negative column
        [[0, 1], [7]],                          # length 1
        [[0, 1], list(range(65))],              # length 65
    ]
    for chroms in bad_cases:
        lens = [len(c) for c in chroms]
        off = torch.tensor(np.concatenate([[0], np.cumsum(lens)]).astype(np.int32), device=dev)
        ci = torch.tensor(np.concatenate(chroms).astype(np.int32), device=dev)
        outs = _outs(torch, len(chroms), dev)
        with pytest.raises(ebic.EbicError) as e:
            ebic.ebic_eval_population_noalloc(x_cm, ci, off, p, *outs)
        assert e.value.code == ebic.EBIC_EINVAL and "invalid chromosome" in str(e.value), chroms
    n = len(off_ok) - 1
    outs = _outs(torch, n, dev)
    ebic.ebic_eval_population_noalloc(x_cm, torch.from_numpy(ci_ok).to(dev),
                                      torch.from_numpy(off_ok).to(dev), p, *outs)
    with ebic.Context(0) as ctx:
        ctx.load_matrix(x)
        want = ctx.eval_population(ci_ok, off_ok, p)
    assert _same([o.cpu().numpy() for o in outs], want)


def test_noalloc_binding_checks_arguments_without_converting(ebic):
    """A wrong dtype, shape, device or length raises before the library is called; nothing is
    converted, because a conversion would allocate."""
    torch = pytest.importorskip("torch")
    dev = torch.device("cuda:0")
    p = ebic.Params.make()
    x, ci_np, off_np = make_inputs(3, 100, 10, 8)
    n = len(off_np) - 1
    x_cm = torch.from_numpy(np.ascontiguousarray(x.T)).to(dev)
    ci, off = torch.from_numpy(ci_np).to(dev), torch.from_numpy(off_np).to(dev)
    good = _outs(torch, n, dev)
    bad = [
        dict(x_colmajor=x_cm.double()),
        dict(x_colmajor=x_cm.reshape(-1)),
        dict(x_colmajor=x_cm.t()),                                  # not contiguous
        dict(col_idx=ci.long()),
        dict(col_idx=ci[:-1]),                                      # shorter than offsets[-1]
        dict(offsets=off.reshape(1, -1)),
        dict(offsets=off.cpu()),
        dict(rows_pos=good[0][:-1]),
        dict(rows_any=good[2].long()),
        dict(fitness=good[3].int()),
        dict(fitness=torch.zeros(n, dtype=torch.int64)),            # host tensor
    ]
    for change in bad:
        kw = dict(x_colmajor=x_cm, col_idx=ci, offsets=off, rows_pos=good[0], rows_neg=good[1],
                  rows_any=good[2], fitness=good[3])
        kw.update(change)
        with pytest.raises(ebic.EbicError) as e:
            ebic.ebic_eval_population_noalloc(params=p, **kw)
        assert e.value.code == ebic.EBIC_EINVAL, list(change)
