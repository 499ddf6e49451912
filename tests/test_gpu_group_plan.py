"""GPU parity of the grouped-product plan (smf_group_plan_*): the batch's host
work done once, its launches captured in a CUDA graph and replayed, with the
launch configuration fixed by flags or chosen by the autotuner's measurements.

Every configuration the autotuner may pick (a narrow shared A at its natural
digit count or padded to three digits; the L2 prefetch ahead of the loads; a
one-digit A in the one-digit kernel's own launch; tiles ordered by K or by MMA
work) is run against the oracle's schoolbook product, and so is every replay
after the operands' contents change in place.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2605_19254_gb300 import inputs  # noqa: E402

FORMS = {"fp64": 0, "limb": 1}

# (M, K, N, bits of A): 7-bit A needs one digit, 12-bit two, 20-bit three (all
# shared across primes); 0 = full 64-bit words, reduced per prime; K = 0 and
# empty products included
SHAPES = [(32, 32, 16, 7), (100, 100, 40, 20), (129, 129, 64, 7), (300, 257, 9, 20), (33, 64, 128, 12),
          (64, 500, 70, 7), (1, 5, 3, 20), (0, 10, 3, 7), (40, 0, 5, 20), (70, 90, 33, 0)]


def dev(words: np.ndarray):
    return torch.from_numpy(np.ascontiguousarray(words).view(np.int64)).cuda()


def host_words(t) -> np.ndarray:
    return t.cpu().numpy().view(np.uint64)


@pytest.fixture(scope="module")
def smf():
    from paper_2605_19254_gb300 import build, smf as _smf
    build.build()
    assert torch.cuda.is_available()
    return _smf


def _operands(seed, shapes):
    out = []
    for i, (M, K, N, ab) in enumerate(shapes):
        if ab:
            A = inputs.rns_matmul_workload(seed + i, M, K, N, ab, 1)[0]
        else:
            A = inputs.random_words(seed + i, "pA", (M, K), 1)
        B = inputs.random_words(seed + i, "pB", (K, N), 8)
        out.append((A, B))
    return out


def _wc(ab, K):
    return ((ab or 63) + 511 + int(np.ceil(np.log2(max(K, 2)))) + 2 + 63) // 64


@pytest.mark.parametrize("form", list(FORMS))
@pytest.mark.parametrize("flags", ["fixed", "pad_all", "prefetch", "one_digit", "order_work",
                                   "pad_all+prefetch+order_work", "one_digit+prefetch+order_work", "autotune"])
def test_plan_matches_oracle_and_replays(smf, orc, form, flags):
    f = {"fixed": 0, "pad_all": smf.SMF_PLAN_PAD_ALL, "prefetch": smf.SMF_PLAN_PREFETCH,
         "order_work": smf.SMF_PLAN_ORDER_WORK,
         "pad_all+prefetch+order_work": smf.SMF_PLAN_PAD_ALL | smf.SMF_PLAN_PREFETCH | smf.SMF_PLAN_ORDER_WORK,
         "one_digit": smf.SMF_PLAN_ONE_DIGIT,
         "one_digit+prefetch+order_work": smf.SMF_PLAN_ONE_DIGIT | smf.SMF_PLAN_PREFETCH | smf.SMF_PLAN_ORDER_WORK,
         "autotune": smf.SMF_PLAN_AUTOTUNE}[flags]
    c = smf.Context(0, FORMS[form])
    bits = [ab for _, _, _, ab in SHAPES]
    ops = _operands(200, SHAPES)
    As = [dev(A) for A, _ in ops]
    Bs = [dev(B) for _, B in ops]
    Cs = [torch.full((M, N, _wc(ab, K)), 7, dtype=torch.int64, device="cuda") for M, K, N, ab in SHAPES]
    plan = c.group_plan(As, Bs, Cs, a_bits=bits, flags=f)
    info = plan.info()
    assert info["graph"] == (form == "limb")
    if form == "limb" and flags.startswith("pad_all"):
        # the 7- and 12-bit products with K > 0 and a non-empty output
        assert info["padded"] == sum(1 for M, K, N, ab in SHAPES if ab in (7, 12) and M and N and K)
    if form == "limb" and flags.startswith("one_digit"):
        # the 7-bit products with K > 0 and a non-empty output
        assert info["one_digit"] == sum(1 for M, K, N, ab in SHAPES if ab == 7 and M and N and K)
    if form == "limb" and "prefetch" in flags:
        assert info["prefetched"] == sum(1 for M, K, N, ab in SHAPES if M and N and K)
    if form == "limb" and "order_work" in flags:
        assert info["tile_order"] == 1
    # the first launch, then two more after new operand contents are copied in
    for rnd, seed in enumerate((200, 400, 600)):
        if rnd:
            ops = _operands(seed, SHAPES)
            for t, (A, B) in zip(As, ops):
                t.copy_(dev(A))
            for t, (_, B) in zip(Bs, ops):
                t.copy_(dev(B))
        for C in Cs:
            C.fill_(7)  # every output is rewritten by each launch
        plan.launch()
        c.status_sync()
        for i, ((M, K, N, ab), (A, B), C) in enumerate(zip(SHAPES, ops, Cs)):
            want = orc.matmul(A, B, _wc(ab, K))
            assert np.array_equal(host_words(C), want), f"launch {rnd}, product {i} {(M, K, N, ab)}"
    plan.destroy()
    c.destroy()


def test_plan_equals_grouped_call_and_survives_its_context(smf):
    # the plan's output is the grouped call's, and a plan may be freed after its context
    c = smf.Context(0, smf.SMF_FORM_INT8LIMB)
    bits = [ab for _, _, _, ab in SHAPES]
    ops = _operands(800, SHAPES)
    As = [dev(A) for A, _ in ops]
    Bs = [dev(B) for _, B in ops]
    C1 = [torch.zeros((M, N, _wc(ab, K)), dtype=torch.int64, device="cuda") for M, K, N, ab in SHAPES]
    C2 = [torch.zeros_like(t) for t in C1]
    c.rns_matmul_grouped(As, Bs, C1, a_bits=bits)
    c.profile_enable(True)  # a graph replays no profiling events: the plan must not record any
    plan = c.group_plan(As, Bs, C2, a_bits=bits)
    plan.launch()
    c.status_sync()
    c.profile_read()
    for a, b in zip(C1, C2):
        assert torch.equal(a, b)
    c.destroy()
    plan.destroy()


def test_plan_autotune_measures_once_per_class(smf, orc):
    # narrow-A classes are measured by the first plan; a second plan of the same
    # shapes on the same context takes every choice from the context's record
    shapes = [(256, 256, 128, 7), (200, 256, 128, 7), (512, 512, 128, 7), (512, 500, 128, 20), (96, 96, 128, 12)]
    bits = [ab for _, _, _, ab in shapes]
    c = smf.Context(0, smf.SMF_FORM_INT8LIMB)
    ops = _operands(900, shapes)
    As = [dev(A) for A, _ in ops]
    Bs = [dev(B) for _, B in ops]
    Cs = [torch.zeros((M, N, _wc(ab, K)), dtype=torch.int64, device="cuda") for M, K, N, ab in shapes]
    p1 = c.group_plan(As, Bs, Cs, a_bits=bits, flags=smf.SMF_PLAN_AUTOTUNE)
    i1 = p1.info()
    # classes: (7-bit, K <= 2^8, M <= 2^8), (7-bit, 2^9, 2^9), (20-bit, 2^9, 2^9), (12-bit, 2^7, 2^7)
    assert i1["classes_tuned"] == 4 and i1["classes_cached"] == 0
    assert p1.report().count("class ") == 4
    p2 = c.group_plan(As, Bs, Cs, a_bits=bits, flags=smf.SMF_PLAN_AUTOTUNE)
    i2 = p2.info()
    assert i2["classes_tuned"] == 0 and i2["classes_cached"] == 4
    assert i2["padded"] == i1["padded"] and i2["prefetched"] == i1["prefetched"]
    for p in (p1, p2):
        for C in Cs:
            C.fill_(7)
        p.launch()
        c.status_sync()
        for (M, K, N, ab), (A, B), C in zip(shapes, ops, Cs):
            assert np.array_equal(host_words(C), orc.matmul(A, B, _wc(ab, K)))
    p1.destroy()
    p2.destroy()
    c.destroy()


def test_plan_autotuned_batched_workload_sampled(smf, orc):
    # the 512-product batch (n log-uniform in [32, 1024], k = 7 / 20, B n x 128 of
    # 512 bits) through an autotuned plan, replayed twice; sampled entries of the
    # smallest, the largest and a spread of other products against the oracle
    batch = inputs.batched_workload(0, 512, 128, 8)
    c = smf.Context(0, smf.SMF_FORM_INT8LIMB)
    As, Bs, Cs, bits, Wcs = [], [], [], [], []
    for n, k, A, B in batch:
        Wc = (k + 511 + int(np.ceil(np.log2(n))) + 2 + 63) // 64
        As.append(dev(A))
        Bs.append(dev(B))
        Cs.append(torch.full((n, 128, Wc), 7, dtype=torch.int64, device="cuda"))
        bits.append(k)
        Wcs.append(Wc)
    plan = c.group_plan(As, Bs, Cs, a_bits=bits, flags=smf.SMF_PLAN_AUTOTUNE)
    assert plan.info()["classes_tuned"] >= 1
    for C in Cs:
        C.fill_(7)
    plan.launch()
    plan.launch()
    c.status_sync()
    ns = [b[0] for b in batch]
    rng = np.random.default_rng(2)
    picks = sorted({int(np.argmin(ns)), int(np.argmax(ns)), 0, 1, 511, *rng.choice(512, 6, replace=False).tolist()})
    for i in picks:
        n, k, A, B = batch[i]
        rows = np.unique(np.append(rng.choice(n, min(n, 4), replace=False), n - 1))
        cols = np.unique(np.append(rng.choice(128, 4, replace=False), 127))
        want = orc.matmul(A[rows], B[:, cols], Wcs[i])
        got = host_words(Cs[i])[rows][:, cols]
        assert np.array_equal(got, want), f"product {i} (n={n}, k={k})"
    plan.destroy()
    c.destroy()


@pytest.mark.parametrize("form", list(FORMS))
def test_plan_of_nothing(smf, form):
    # no products, or only empty ones: the plan launches nothing and writes nothing
    c = smf.Context(0, FORMS[form])
    p = c.group_plan([], [], [], flags=smf.SMF_PLAN_AUTOTUNE)
    p.launch()
    p.destroy()
    A = torch.zeros((0, 5, 1), dtype=torch.int64, device="cuda")
    B = torch.zeros((5, 3, 8), dtype=torch.int64, device="cuda")
    C = torch.zeros((0, 3, 10), dtype=torch.int64, device="cuda")
    p = c.group_plan([A], [B], [C], a_bits=7, flags=smf.SMF_PLAN_AUTOTUNE)
    p.launch()
    c.status_sync()
    assert p.info()["padded"] == 0
    p.destroy()
    c.destroy()
