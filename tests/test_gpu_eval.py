"""GPU parity of population evaluation against the CPU oracle, through the C ABI.

Bar: bit-exact (counts and fitness are integers; comparisons of float32 values are exact on both
sides), for every evaluation form (direct, bitmap, plain one-launch-per-individual, auto)."""

import numpy as np
import pytest

from oracle import counts as ocounts
from oracle.bitmap import pair_bitmap
from oracle.params import Params as OParams
from paper_2105_01196_gb300 import synth

pytestmark = pytest.mark.gpu

MODES = (1, 2, 3, 4, 0)  # direct, bitmap, plain, staged, auto


@pytest.fixture(scope="module")
def ebic():
    from paper_2105_01196_gb300 import ebic as e
    return e


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return torch


def oparams(neg, num, den, min_rows=2, col_cap=10, ns=0, lk=0):
    return OParams(neg_trends=neg, ratio_num=num, ratio_den=den, min_rows=min_rows,
                   col_cap=col_cap, non_strict=ns, last_kept=lk)


def oracle_eval(x, col_idx, offsets, neg, num, den, sample=None, min_rows=2, col_cap=10, ns=0,
                lk=0):
    p = oparams(neg, num, den, min_rows, col_cap, ns, lk)
    n = len(offsets) - 1
    idx = range(n) if sample is None else sample
    out = {}
    for i in idx:
        cols = [int(c) for c in col_idx[offsets[i]:offsets[i + 1]]]
        out[i] = ocounts.eval_individual(x, cols, p)
    return out


def assert_parity(got, want):
    rp, rn, ra, f = (np.asarray(a) for a in got)
    for i, (wp, wn, wa, wf) in want.items():
        assert (int(rp[i]), int(rn[i]), int(ra[i]), int(f[i])) == (wp, wn, wa, wf), \
            f"individual {i}: got {(rp[i], rn[i], ra[i], f[i])} want {(wp, wn, wa, wf)}"


def test_tiny_workload_all_modes(ebic):
    x, _, ci, off = synth.workload_inputs(synth.WORKLOADS["tiny"])
    with ebic.Context(0) as ctx:
        ctx.load_matrix(x)
        for neg in (0, 1):
            for num, den in ((1, 1), (85, 100), (1, 2)):
                want = oracle_eval(x, ci, off, neg, num, den)
                for mode in MODES:
                    p = ebic.Params.make(neg_trends=neg, ratio_num=num, ratio_den=den, mode=mode)
                    assert_parity(ctx.eval_population(ci, off, p), want)


def ragged_population(g, n, C, lens=None):
    if lens is None:
        lens = g.integers(2, min(64, C) + 1, size=n)
    lens = np.asarray(lens)
    off = np.zeros(len(lens) + 1, np.int32)
    off[1:] = np.cumsum(lens)
    ci = np.concatenate([g.choice(C, size=int(L), replace=False) for L in lens]).astype(np.int32)
    return ci, off


@pytest.mark.parametrize("R,C", [(1, 2), (31, 3), (32, 17), (33, 64), (127, 65), (129, 7),
                                 (1000, 20), (4097, 40)])
def test_ragged_shapes_ties_and_zeros(ebic, R, C):
    g = np.random.default_rng(R * 1000 + C)
    x = (g.integers(-2, 3, size=(R, C)) * 0.5).astype(np.float32)
    x[g.random((R, C)) < 0.05] = -0.0
    x[g.random((R, C)) < 0.02] = np.float32(1e-42)
    lens = [2, min(64, C)] + list(g.integers(2, min(64, C) + 1, size=40))
    ci, off = ragged_population(g, len(lens), C, lens)
    with ebic.Context(0) as ctx:
        ctx.load_matrix(x)
        for neg, num, den in ((1, 1, 1), (1, 85, 100), (0, 2, 3)):
            want = oracle_eval(x, ci, off, neg, num, den, min_rows=0)
            for mode in MODES:
                p = ebic.Params.make(neg_trends=neg, ratio_num=num, ratio_den=den, mode=mode,
                                     min_rows=0)
                assert_parity(ctx.eval_population(ci, off, p), want)


def test_default_workload_full_parity(ebic):
    w = synth.WORKLOADS["default"]
    x, _, ci, off = synth.workload_inputs(w)
    want = oracle_eval(x, ci, off, 1, 85, 100)
    with ebic.Context(0) as ctx:
        ctx.load_matrix(x)
        for mode in MODES:
            p = ebic.Params.make(neg_trends=1, ratio_num=85, ratio_den=100, mode=mode)
            assert_parity(ctx.eval_population(ci, off, p), want)


@pytest.mark.parametrize("name,n_sample", [("batched", 160), ("tieheavy", 48)])
def test_large_workloads_sampled(ebic, name, n_sample):
    w = synth.WORKLOADS[name]
    x, _, ci, off = synth.workload_inputs(w)
    g = np.random.default_rng(5)
    n = len(off) - 1
    lens = np.diff(off)
    sample = sorted(set(g.choice(n, size=n_sample, replace=False).tolist())
                    | {int(np.argmax(lens)), int(np.argmin(lens)), n - 1})
    with ebic.Context(0) as ctx:
        ctx.load_matrix(x)
        for neg, num, den in ((1, 85, 100), (1, 1, 1)):
            want = oracle_eval(x, ci, off, neg, num, den, sample=sample)
            for mode in (1, 2, 4):
                p = ebic.Params.make(neg_trends=neg, ratio_num=num, ratio_den=den, mode=mode)
                assert_parity(ctx.eval_population(ci, off, p), want)


def test_device_pointers_and_col_major(ebic, torch_cuda):
    torch = torch_cuda
    g = np.random.default_rng(9)
    x = g.standard_normal((5000, 30)).astype(np.float32)
    ci, off = ragged_population(g, 300, 30)
    want = oracle_eval(x, ci, off, 1, 85, 100)
    dev = torch.device("cuda:0")
    with ebic.Context(0, torch.cuda.current_stream().cuda_stream) as ctx:
        for layout, xin in ((ebic.ROW_MAJOR, torch.from_numpy(x).to(dev)),
                            (ebic.COL_MAJOR, torch.from_numpy(np.ascontiguousarray(x.T)).to(dev)),
                            (ebic.COL_MAJOR, np.ascontiguousarray(x.T))):
            ctx.load_matrix(xin, layout)
            for mode in (1, 2, 3, 4):
                p = ebic.Params.make(neg_trends=1, ratio_num=85, ratio_den=100, mode=mode)
                outs = [torch.zeros(300, dtype=torch.int32, device=dev) for _ in range(3)]
                outs.append(torch.zeros(300, dtype=torch.int64, device=dev))
                ctx.eval_population(torch.from_numpy(ci).to(dev), torch.from_numpy(off).to(dev),
                                    p, *outs)
                got = [o.cpu().numpy() for o in outs]
                assert_parity(got, want)


@pytest.mark.parametrize("values", ["ties", "distinct"])
@pytest.mark.parametrize("R,C", [(77, 2), (300, 3), (130, 5), (1030, 9), (200, 16),
                                 (64, 17), (40, 33), (33, 64), (257, 65), (129, 128),
                                 (100, 129), (97, 256), (70, 257), (35, 512), (66, 513),
                                 (45, 1000), (33, 1024), (40, 1025)])
def test_bitmap_matches_oracle_definition(ebic, R, C, values):
    """Every pair word against the oracle's definition: from the bit planes of the rank codes up
    to 1,024 columns (1 to 10 planes) and the order-key build beyond; values -3..3 (many ties)
    or distinct ones, with signed zeros, subnormals and extreme magnitudes; rows not a multiple
    of 32.  Up to 129 columns every pair is compared, beyond that a sample that includes the
    first, last and diagonal pairs."""
    from oracle.bitmap import pair_words
    g = np.random.default_rng(11 + R * 3 + C + (values == "distinct"))
    if values == "ties":
        x = g.integers(-3, 4, size=(R, C)).astype(np.float32)
    else:
        x = g.standard_normal((R, C)).astype(np.float32)
    x[g.random((R, C)) < 0.05] = -0.0
    x[g.random((R, C)) < 0.02] = np.float32(1e-45)
    x[g.random((R, C)) < 0.02] = -np.float32(3e-42)
    x[g.random((R, C)) < 0.01] = np.finfo(np.float32).max
    x[g.random((R, C)) < 0.01] = -np.finfo(np.float32).max
    W = (R + 31) // 32
    with ebic.Context(0) as ctx:
        ctx.load_matrix(x)
        ctx.build_bitmap()
        wst = ((R + 127) // 128) * 4
        out = np.zeros(C * C * wst, np.uint32)
        ctx.copy_bitmap(out)
        got = out.reshape(C, C, wst)
    assert not got[:, :, W:].any()
    if C <= 129:
        assert np.array_equal(got[:, :, :W], pair_bitmap(x))
        return
    pairs = {(0, 1), (1, 0), (0, C - 1), (C - 1, 0), (C - 2, C - 1), (C - 1, C - 2), (5, 5),
             (C - 1, C - 1)}
    pairs |= {(int(a), int(b)) for a, b in g.integers(0, C, size=(300, 2))}
    for a, b in sorted(pairs):
        assert np.array_equal(got[a, b, :W], pair_words(x, a, b)), (a, b)


@pytest.mark.parametrize("D", [1, 2, 3, 4, 5, 9, 17, 33, 129, 257, 513, 1000])
def test_bitmap_rows_of_few_distinct_values(ebic, D):
    """Rows that hold at most D distinct values (one row all D of them; D at the bit boundaries
    of D - 1, a constant matrix at D = 1): pair words of a sample of pairs and their pair counts
    against the oracle."""
    from oracle.bitmap import pair_words
    g = np.random.default_rng(900 + D)
    C = max(D + 3, 4) if D < 1000 else 1000
    R = 300
    levels = np.sort(g.standard_normal(D)).astype(np.float32)
    x = levels[g.integers(0, D, size=(R, C))]
    x[0, :D] = levels[g.permutation(D)]  # (row 0 holds every level)
    W = (R + 31) // 32
    with ebic.Context(0) as ctx:
        ctx.load_matrix(x)
        ctx.build_bitmap()
        wst = ((R + 127) // 128) * 4
        out = np.zeros(C * C * wst, np.uint32)
        ctx.copy_bitmap(out)
        cnt = np.zeros(C * C, np.uint64)
        ctx.copy_pair_counts(cnt)
    got = out.reshape(C, C, wst)
    cnt = cnt.reshape(C, C)
    popc = lambda w: int(np.unpackbits(np.asarray(w, np.uint32).view(np.uint8)).sum())
    pairs = {(0, 1), (0, C - 1), (C - 2, C - 1)}
    pairs |= {tuple(sorted((int(a), int(b)))) for a, b in g.integers(0, C, size=(200, 2)) if a != b}
    for a, b in sorted(pairs):
        wab, wba = pair_words(x, a, b), pair_words(x, b, a)
        assert np.array_equal(got[a, b, :W], wab) and np.array_equal(got[b, a, :W], wba), (a, b)
        assert int(cnt[a, b]) == popc(wab) | (popc(wba) << 32), (a, b)
    assert not got[:, :, W:].any()


@pytest.mark.parametrize("R,C", [(1, 2), (33, 7), (300, 129), (129, 200), (40, 1000)])
def test_pair_counts_match_oracle_words(ebic, R, C):
    """The pair counts the plane build accumulates (one 64-bit atomic per pair and 32-word
    chunk): for a < b, the popcounts of the oracle's pair words G[a][b] and G[b][a] in the low and
    high halves, zero elsewhere; on a tie-heavy matrix with rows not a multiple of 32."""
    from oracle.bitmap import pair_words
    g = np.random.default_rng(5 + R + C)
    x = g.integers(-2, 3, size=(R, C)).astype(np.float32)
    with ebic.Context(0) as ctx:
        ctx.load_matrix(x)
        ctx.build_bitmap()
        out = np.zeros(C * C, np.uint64)
        ctx.copy_pair_counts(out)
    t = out.reshape(C, C)
    assert not np.tril(t).any()
    pairs = [(a, b) for a in range(C) for b in range(a + 1, C)]
    if len(pairs) > 4000:
        idx = g.choice(len(pairs), 4000, replace=False)
        pairs = [pairs[i] for i in idx] + [(0, 1), (0, C - 1), (C - 2, C - 1)]
    popc = lambda w: int(np.unpackbits(np.asarray(w, np.uint32).view(np.uint8)).sum())
    for a, b in pairs:
        lo, hi = int(t[a, b]) & 0xFFFFFFFF, int(t[a, b]) >> 32
        assert (lo, hi) == (popc(pair_words(x, a, b)), popc(pair_words(x, b, a))), (a, b)


def test_errors_are_reported(ebic, torch_cuda):
    torch = torch_cuda
    x = np.ones((10, 4), np.float32)
    with ebic.Context(0) as ctx:
        p = ebic.Params.make()
        with pytest.raises(ebic.EbicError) as e:
            ctx.eval_population(np.array([0, 1], np.int32), np.array([0, 2], np.int32), p)
        assert e.value.code == ebic.EBIC_ESTATE
        for bad in (np.nan, np.inf, -np.inf):
            y = x.copy()
            y[3, 2] = bad
            with pytest.raises(ebic.EbicError) as e:
                ctx.load_matrix(y)
            assert e.value.code == ebic.EBIC_ENAN
        ctx.load_matrix(x)
        bad_pops = [([0, 0], [0, 2]), ([0], [0, 1]), ([0, 4], [0, 2]), ([-1, 2], [0, 2]),
                    (list(range(4)) * 17, [0, 68])]
        for cols, offs in bad_pops:
            for dev in (False, True):
                c = np.array(cols, np.int32)
                o = np.array(offs, np.int32)
                if dev:
                    c, o = torch.from_numpy(c).cuda(), torch.from_numpy(o).cuda()
                with pytest.raises(ebic.EbicError) as e:
                    ctx.eval_population(c, o, p)
                assert e.value.code == ebic.EBIC_EINVAL
        with pytest.raises(ebic.EbicError) as e:
            ctx.eval_population(np.array([0, 1], np.int32), np.array([0, 2], np.int32),
                                ebic.Params.make(ratio_num=0))
        assert e.value.code == ebic.EBIC_EINVAL
        r = ctx.eval_population(np.zeros(0, np.int32), np.zeros(1, np.int32), p)
        assert all(len(a) == 0 for a in r)
        # the context stays usable after every error
        r = ctx.eval_population(np.array([0, 1], np.int32), np.array([0, 2], np.int32), p)
        assert int(r[2][0]) == 0


@pytest.mark.parametrize("R,C", [(700, 128), (700, 129), (520, 1024), (300, 1025)])
def test_code_width_boundaries(ebic, R, C):
    """The direct form reads 8-bit per-row rank codes up to 128 columns, 16-bit ones up to 1,024
    and the 32-bit order keys beyond; each width against the oracle, on tie-heavy values with
    signed zeros and extreme magnitudes, rows not a multiple of the kernel's pass."""
    g = np.random.default_rng(R * 7 + C)
    x = g.integers(-3, 4, size=(R, C)).astype(np.float32)
    x[g.random((R, C)) < 0.05] = -0.0
    x[g.random((R, C)) < 0.01] = np.finfo(np.float32).max
    x[g.random((R, C)) < 0.01] = -np.finfo(np.float32).max
    x[g.random((R, C)) < 0.01] = np.float32(1e-45)
    x[: R // 10] = 1.5                              # rows of one value: no trend at all
    ci, off = ragged_population(g, 48, C)
    with ebic.Context(0) as ctx:
        ctx.profile_enable(True)
        ctx.load_matrix(x)
        assert ctx.profile_read(ebic.KERNEL_RANK_CODES)["launches"] == 0  # built on first use
        for neg, num, den in ((1, 85, 100), (0, 1, 1), (1, 1, 2)):
            want = oracle_eval(x, ci, off, neg, num, den)
            for mode in (1, 2, 4):
                p = ebic.Params.make(neg_trends=neg, ratio_num=num, ratio_den=den, mode=mode)
                assert_parity(ctx.eval_population(ci, off, p), want)
        st = ctx.profile_read(ebic.KERNEL_RANK_CODES)
        assert st["launches"] == (1 if C <= 1024 else 0)


def tie_matrix(g, R, C):
    x = g.integers(-3, 4, size=(R, C)).astype(np.float32)
    x[g.random((R, C)) < 0.05] = -0.0
    x[: R // 10] = 1.5                              # rows of one value
    return x


@pytest.mark.parametrize("R,C", [(200, 20), (700, 129), (300, 1025)])
def test_trend_variants_all_forms(ebic, R, C):
    """Ties counting for both directions (non_strict) and counting against the last kept value
    (last_kept), each form against the oracle: 8-bit codes, 16-bit codes and order keys for the
    direct form, the bitmap (non_strict only), the plain form; rows not a multiple of 32."""
    g = np.random.default_rng(R + C)
    x = tie_matrix(g, R, C)
    ci, off = ragged_population(g, 40, C)
    with ebic.Context(0) as ctx:
        ctx.load_matrix(x)
        for ns, lk in ((1, 0), (0, 1), (1, 1)):
            for neg, num, den in ((1, 1, 1), (1, 85, 100), (0, 1, 2)):
                want = oracle_eval(x, ci, off, neg, num, den, ns=ns, lk=lk)
                for mode in (1, 2, 3, 4, 0):
                    p = ebic.Params.make(neg_trends=neg, ratio_num=num, ratio_den=den, mode=mode,
                                         non_strict=ns, last_kept=lk)
                    if mode == 2 and lk:
                        with pytest.raises(ebic.EbicError) as e:
                            ctx.eval_population(ci, off, p)
                        assert e.value.code == ebic.EBIC_EINVAL
                        continue
                    assert_parity(ctx.eval_population(ci, off, p), want)


def test_trend_variants_default_workload(ebic):
    w = synth.WORKLOADS["default"]
    x, _, ci, off = synth.workload_inputs(w)
    g = np.random.default_rng(4)
    sample = sorted(g.choice(len(off) - 1, size=120, replace=False).tolist())
    with ebic.Context(0) as ctx:
        ctx.load_matrix(x)
        for ns, lk in ((1, 0), (0, 1)):
            want = oracle_eval(x, ci, off, 1, 85, 100, sample=sample, ns=ns, lk=lk)
            for mode in ((1, 2, 0) if not lk else (1, 0)):
                p = ebic.Params.make(neg_trends=1, ratio_num=85, ratio_den=100, mode=mode,
                                     non_strict=ns, last_kept=lk)
                assert_parity(ctx.eval_population(ci, off, p), want)


def test_bitmap_larger_than_l2_all_variants(ebic, torch_cuda):
    """A pair bitmap larger than the device's L2 (243 MB), which the bitmap kernel reads through
    its shared-memory staging for ratios below 1 (exact items included: short chromosomes at
    ratio 0.85) and with register rounds at ratio 1: both directions and one, ties for both
    directions or not; chromosomes of 2 to 64 columns (one to several staged batches of pairs);
    4,500 rows (the last pass of 128 words only partly filled, pad rows in the last word)."""
    R, C = 4500, 650
    bitmap_bytes = C * C * ((R + 127) // 128 * 128 // 32) * 4
    l2 = getattr(torch_cuda.cuda.get_device_properties(0), "L2_cache_size", 0)
    assert l2 == 0 or bitmap_bytes > l2
    g = np.random.default_rng(77)
    x = tie_matrix(g, R, C)
    lens = np.concatenate([[2, 3, 13, 14, 25, 26, 64], g.integers(2, 65, size=33)])
    ci, off = ragged_population(g, len(lens), C, lens)
    with ebic.Context(0) as ctx:
        ctx.load_matrix(x)
        for neg, ns in ((1, 0), (1, 1), (0, 0), (0, 1)):
            for num, den in ((85, 100), (1, 1), (1, 2)):
                want = oracle_eval(x, ci, off, neg, num, den, ns=ns)
                p = ebic.Params.make(neg_trends=neg, ratio_num=num, ratio_den=den, mode=2,
                                     non_strict=ns)
                assert_parity(ctx.eval_population(ci, off, p), want)


@pytest.mark.parametrize("ipw", [2, 3, 4])
def test_staged_groups_of_individuals(ebic, torch_cuda, ipw):
    """The staged bitmap form with 2, 3 or 4 individuals per work item (the last group partial
    when the population is not a multiple): one stream of staged units across the group's
    individuals, dead-free CSR individuals of 2 to 64 columns (single and several units per
    pass), both directions and one, ties counting both ways or not, against the oracle."""
    R, C = 4500, 650
    g = np.random.default_rng(91 + ipw)
    x = tie_matrix(g, R, C)
    lens = np.concatenate([[2, 2, 3, 7, 8, 13, 14, 64], g.integers(2, 65, size=27)])
    ci, off = ragged_population(g, len(lens), C, lens)
    with ebic.Context(0) as ctx:
        ctx.load_matrix(x)
        for neg, ns in ((1, 0), (1, 1), (0, 0)):
            for num, den in ((85, 100), (1, 2)):
                want = oracle_eval(x, ci, off, neg, num, den, ns=ns)
                p = ebic.Params.make(neg_trends=neg, ratio_num=num, ratio_den=den, mode=2,
                                     non_strict=ns, ipw=ipw)
                assert_parity(ctx.eval_population(ci, off, p), want)
        with pytest.raises(ebic.EbicError):
            ctx.eval_population(ci, off, ebic.Params.make(ipw=5))


def test_csr_validation_long_chromosomes(ebic):
    """Repeated columns are rejected wherever they sit in a chromosome of up to 64 columns (both
    within the first 32, both within the last 32, one in each), and one bad individual among
    valid ones rejects the call; a valid 64-column individual passes."""
    g = np.random.default_rng(8)
    x = g.standard_normal((300, 100)).astype(np.float32)
    good = [list(g.choice(100, size=L, replace=False)) for L in (64, 40, 33, 2)]
    with ebic.Context(0) as ctx:
        ctx.load_matrix(x)
        p = ebic.Params.make(neg_trends=1, ratio_num=1, ratio_den=2)

        def csr(pop):
            off = np.concatenate([[0], np.cumsum([len(c) for c in pop])]).astype(np.int32)
            return np.concatenate(pop).astype(np.int32), off

        ci, off = csr(good)
        want = oracle_eval(x, ci, off, 1, 1, 2)
        assert_parity(ctx.eval_population(ci, off, p), want)
        for a, b in ((0, 31), (33, 50), (3, 35), (31, 32), (0, 63)):
            bad = list(good[0])
            bad[b] = bad[a]
            ci, off = csr(good[1:] + [bad])
            with pytest.raises(ebic.EbicError) as e:
                ctx.eval_population(ci, off, p)
            assert e.value.code == ebic.EBIC_EINVAL
