"""GPU tests of the ensemble path (kpm_moments_batch / kpm_batch_*): every
problem of a batch must give the moments the single-problem path and the
FP64 oracle give, with uneven sizes, moment counts and block widths in one
graph launch."""
import numpy as np
import pytest

from kpm_inputs import hamiltonians as ham
from kpm_inputs import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def kpm():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1410_5242_gb300 import build
    build.build()
    from paper_1410_5242_gb300 import kpm as k
    return k


def problems():
    """Uneven little ensemble: lattices of several shapes, one open boundary,
    one ragged random matrix; M from 2 to 130; R from 1 to 64."""
    return [
        (ham.ti_hamiltonian(5, 4, 3, gamma=0.5, seed=1), 64, 8, 11),
        (ham.ti_hamiltonian(6, 6, 6, gamma=2.0, seed=2), 130, 32, 12),
        (ham.ti_hamiltonian(3, 4, 7, gamma=1.0, seed=3, periodic=(True, True, False)), 40, 16, 13),
        (ham.random_hermitian(203, 7, seed=4, empty_rows=0.1), 96, 64, 14),
        (ham.ti_hamiltonian(4, 4, 4, gamma=0.0), 2, 4, 15),
        (ham.ti_hamiltonian(3, 3, 3, gamma=3.0, seed=5), 18, 1, 16),
        (ham.ti_hamiltonian(7, 3, 3, gamma=0.7, seed=6), 64, 2, 17),
    ]


def contexts(kpm, probs, prec):
    out = []
    for h, M, R, seed in probs:
        a, b = kpm.scale_from_bounds(*kpm.gershgorin(h), 0.01)
        out.append((kpm.create(h, a, b, precision=prec, chunk_height=8, sigma=16), h, a, b))
    return out


@pytest.mark.parametrize("prec", [0, 1])
def test_batch_matches_single_problem_and_oracle(kpm, orc, prec):
    probs = problems()
    ctxs = contexts(kpm, probs, prec)
    etas = kpm.moments_batch([c for c, *_ in ctxs], [p[1] for p in probs], [p[2] for p in probs],
                             [p[3] for p in probs])
    for (ctx, h, a, b), (_, M, R, seed), eta in zip(ctxs, probs, etas):
        single = ctx.moments(M, R, seed)
        ref, _ = orc.moments(h, a, b, M, seed, range(R))
        eta0 = ref[:, :1]
        if prec == 0:
            assert np.all(np.abs(eta - single) <= 1e-12 * eta0)
            assert np.all(np.abs(eta - ref) <= 1e-10 * eta0)
        else:
            assert np.abs(kpm.eta_to_mu(eta) - kpm.eta_to_mu(single)).max() <= 1e-6
            assert np.abs(kpm.eta_to_mu(eta) - orc.eta_to_mu(ref)).max() <= 1e-5
    for c, *_ in ctxs:
        c.close()


@pytest.mark.parametrize("prec", [0, 1])
def test_batch_object_relaunch_is_reproducible(kpm, prec):
    probs = problems()[:4]
    ctxs = contexts(kpm, probs, prec)
    Ms, Rs, seeds = [p[1] for p in probs], [p[2] for p in probs], [p[3] for p in probs]
    with kpm.Batch([c for c, *_ in ctxs], Ms, Rs, seeds) as batch:
        info = batch.info()
        assert info["count"] == 4 and info["steps"] == max(Ms) // 2
        # one phase launch per problem; per step, a sweep and a reduction for
        # each lane-shape class (problems of equal R) that is still running
        class_steps = {}
        for M, R in zip(Ms, Rs):
            class_steps[R] = max(class_steps.get(R, 0), M // 2)
        assert info["kernel_launches"] == 4 + 2 * sum(class_steps.values())
        assert info["sweeps"] == sum(M // 2 for M in Ms)
        batch.launch()
        first = [batch.eta(p) for p in range(4)]
        batch.launch()
        second = [batch.eta(p) for p in range(4)]
    for x, y in zip(first, second):
        assert np.array_equal(x, y)
    for c, *_ in ctxs:
        c.close()


def test_batch_rejects_bad_requests(kpm):
    probs = problems()[:2]
    ctxs = contexts(kpm, probs, 1)
    c0, c1 = ctxs[0][0], ctxs[1][0]
    for Ms, Rs, cs, status in (([64, 30], [8, 0], [c0, c1], kpm.KPM_EINVAL),
                               ([64, 31], [8, 8], [c0, c1], kpm.KPM_EINVAL),
                               ([64, 30], [8, 8], [c0, c0], kpm.KPM_EINVAL)):
        with pytest.raises(kpm.KPMError) as e:
            kpm.moments_batch(cs, Ms, Rs, [1, 2])
        assert e.value.status == status
    h = probs[0][0]
    a, b = kpm.scale_from_bounds(*kpm.gershgorin(h), 0.01)
    with kpm.create(h, a, b, precision=0) as c64:
        with pytest.raises(kpm.KPMError) as e:
            kpm.moments_batch([c0, c64], [8, 8], [8, 8], [1, 2])
        assert e.value.status == kpm.KPM_EINVAL
    for c, *_ in ctxs:
        c.close()


def widths(R):
    """Power-of-two column blocks of at most 64, widest first."""
    out, rest, w = [], R, 64
    while rest:
        while rest >= w:
            out.append(w)
            rest -= w
        w //= 2
    return out


@pytest.mark.parametrize("prec", [0, 1])
def test_batch_any_block_width(kpm, orc, prec):
    """Block widths that are not a power of two, or above 64, are split into
    column blocks that join the classes of their widths (two blocks of one
    problem in one class where R = 128): every problem's moments must equal
    the single-problem path's, which splits the same way, and the oracle's
    on its first, middle and last vectors."""
    probs = [
        (ham.ti_hamiltonian(6, 5, 4, gamma=1.0, seed=31), 40, 48, 41),
        (ham.ti_hamiltonian(5, 5, 5, gamma=0.5, seed=32), 24, 7, 42),
        (ham.ti_hamiltonian(4, 6, 5, gamma=2.0, seed=33), 32, 100, 43),
        (ham.ti_hamiltonian(7, 4, 3, gamma=1.5, seed=34), 16, 128, 44),
        (ham.ti_hamiltonian(3, 3, 4, gamma=0.7, seed=35), 12, 3, 45),
        (ham.ti_hamiltonian(4, 4, 4, gamma=1.0, seed=36), 20, 16, 46),
    ]
    ctxs = contexts(kpm, probs, prec)
    Ms, Rs, seeds = [p[1] for p in probs], [p[2] for p in probs], [p[3] for p in probs]
    with kpm.Batch([c for c, *_ in ctxs], Ms, Rs, seeds) as batch:
        info = batch.info()
        blocks = {}  # width -> longest M among its blocks
        for M, R in zip(Ms, Rs):
            for w in widths(R):
                blocks[w] = max(blocks.get(w, 0), M // 2)
        assert info["count"] == len(probs) and info["classes"] == len(blocks)
        assert info["kernel_launches"] == len(probs) + 2 * sum(blocks.values())
        assert info["sweeps"] == sum(M // 2 for M in Ms)
        if prec == 1:
            assert info["staged_classes"] == sum(1 for w in blocks if w >= 8)
        batch.launch()
        etas = [batch.eta(p) for p in range(len(probs))]
    for (ctx, h, a, b), (_, M, R, seed), eta in zip(ctxs, probs, etas):
        assert eta.shape == (R, M)
        single = ctx.moments(M, R, seed)
        cols = sorted({0, R // 2, R - 1})
        ref, _ = orc.moments(h, a, b, M, seed, cols)
        eta0 = ref[:, :1]
        if prec == 0:
            assert np.all(np.abs(eta - single) <= 1e-12 * np.abs(single[:, :1]))
            assert np.all(np.abs(eta[cols] - ref) <= 1e-10 * eta0)
        else:
            assert np.abs(kpm.eta_to_mu(eta) - kpm.eta_to_mu(single)).max() <= 1e-6
            assert np.abs(kpm.eta_to_mu(eta[cols]) - orc.eta_to_mu(ref)).max() <= 1e-5
    for c, *_ in ctxs:
        c.close()


def test_ensemble_recipe_sampled_against_oracle(kpm, orc):
    """The four smallest lattices of the 64-problem ensemble recipe (complex
    float storage), moments capped at 128 so the oracle finishes quickly;
    vectors 0 and 1 of each checked against the oracle."""
    ens = sorted(workloads.ensemble(), key=lambda p: np.prod(p["dims"]))[:4]
    ctxs, Ms, Rs, seeds = [], [], [], []
    for p in ens:
        h = ham.ti_hamiltonian(*p["dims"], gamma=p["gamma"], seed=p["seed"])
        a, b = kpm.scale_from_bounds(*kpm.gershgorin(h), 0.01)
        ctxs.append((kpm.create(h, a, b, precision=kpm.PREC_FP32), h, a, b))
        Ms.append(min(p["M"], 128))
        Rs.append(p["R"])
        seeds.append(p["seed"])
    etas = kpm.moments_batch([c for c, *_ in ctxs], Ms, Rs, seeds)
    for (ctx, h, a, b), M, seed, eta in zip(ctxs, Ms, seeds, etas):
        ref, _ = orc.moments(h, a, b, M, seed, [0, 1])
        dmu = np.abs(kpm.eta_to_mu(eta[:2]) - orc.eta_to_mu(ref)).max()
        assert dmu <= 1e-5, dmu
        ctx.close()


def test_staged_batch_classes_with_several_problems(kpm, orc):
    """Complex float classes of several problems each (R = 16 and 32) run the
    staged kernel over the concatenated chunks of the running problems; the
    eta flush at every problem boundary must give each problem its own
    moments.  Sizes include a lattice with fewer chunks than blocks and a
    ragged matrix whose rows are not a multiple of the chunk height."""
    probs = [
        (ham.ti_hamiltonian(8, 8, 8, gamma=0.5, seed=1), 80, 16, 21),
        (ham.ti_hamiltonian(3, 3, 3, gamma=1.0, seed=2), 40, 16, 22),
        (ham.random_hermitian(517, 9, seed=3, empty_rows=0.05), 64, 16, 23),
        (ham.ti_hamiltonian(12, 10, 9, gamma=2.5, seed=4), 120, 32, 24),
        (ham.ti_hamiltonian(5, 6, 4, gamma=0.1, seed=5), 24, 32, 25),
        (ham.ti_hamiltonian(16, 16, 8, gamma=1.5, seed=6), 64, 32, 26),
    ]
    ctxs = []
    for h, M, R, seed in probs:
        a, b = kpm.scale_from_bounds(*kpm.gershgorin(h), 0.01)
        ctxs.append((kpm.create(h, a, b, precision=kpm.PREC_FP32), h, a, b))
    for c, *_ in ctxs:
        assert c.get_launch(16)["stages"] >= 1 and c.get_launch(32)["stages"] >= 1
    etas = kpm.moments_batch([c for c, *_ in ctxs], [p[1] for p in probs], [p[2] for p in probs],
                             [p[3] for p in probs])
    etas2 = kpm.moments_batch([c for c, *_ in ctxs], [p[1] for p in probs],
                              [p[2] for p in probs], [p[3] for p in probs])
    for (ctx, h, a, b), (_, M, R, seed), eta, eta2 in zip(ctxs, probs, etas, etas2):
        assert np.array_equal(eta, eta2)
        single = ctx.moments(M, R, seed)
        cols = [0, R - 1]
        ref, _ = orc.moments(h, a, b, M, seed, cols)
        assert np.abs(kpm.eta_to_mu(eta) - kpm.eta_to_mu(single)).max() <= 1e-6
        assert np.abs(kpm.eta_to_mu(eta[cols]) - orc.eta_to_mu(ref)).max() <= 1e-5
    for c, *_ in ctxs:
        c.close()


def test_batch_classes_take_their_first_problems_launch_shape(kpm, orc):
    """A class runs with the launch shape its first problem's context uses
    for the width (kpm_set_launch / kpm_autotune): the register path for one
    class, one stage for another; the moments stay those of the single
    problems."""
    probs = [
        (ham.ti_hamiltonian(8, 8, 6, gamma=0.5, seed=1), 48, 16, 31),
        (ham.ti_hamiltonian(5, 5, 5, gamma=1.0, seed=2), 32, 16, 32),
        (ham.ti_hamiltonian(9, 7, 6, gamma=2.0, seed=3), 40, 32, 33),
        (ham.ti_hamiltonian(6, 6, 6, gamma=0.3, seed=4), 24, 32, 34),
    ]
    ctxs = []
    for h, M, R, seed in probs:
        a, b = kpm.scale_from_bounds(*kpm.gershgorin(h), 0.01)
        ctxs.append((kpm.create(h, a, b, precision=kpm.PREC_FP32), h, a, b))
    # batch order is by width, then by decreasing M: the first problem of
    # each class is the one with the largest M
    ctxs[0][0].set_launch(16, 4, 4, 128, tile_groups=1, stages=0)
    ctxs[2][0].set_launch(32, 8, 4, 128, stages=1)
    b = kpm.Batch([c for c, *_ in ctxs], [p[1] for p in probs], [p[2] for p in probs],
                  [p[3] for p in probs])
    info = b.info()
    b.close()
    assert info["classes"] == 2 and info["staged_classes"] == 1
    etas = kpm.moments_batch([c for c, *_ in ctxs], [p[1] for p in probs], [p[2] for p in probs],
                             [p[3] for p in probs])
    for (ctx, h, a, b), (_, M, R, seed), eta in zip(ctxs, probs, etas):
        ref, _ = orc.moments(h, a, b, M, seed, [0, R - 1])
        assert np.abs(kpm.eta_to_mu(eta[[0, R - 1]]) - orc.eta_to_mu(ref)).max() <= 1e-5
    for c, *_ in ctxs:
        c.close()


def test_smaller_layout_between_batch_launches(kpm):
    """A batch's captured graph keeps launching after another context has
    planned and run the same staged instantiation with a smaller shared-
    memory layout: the occupancy queries and launches only ever raise the
    kernel's dynamic shared-memory limit, so the graph's larger stages stay
    allowed and its moments do not change."""
    big = []
    for h in (ham.ti_hamiltonian(10, 10, 8, gamma=1.0, seed=21),
              ham.ti_hamiltonian(8, 8, 6, gamma=0.5, seed=22)):
        a, b = kpm.scale_from_bounds(*kpm.gershgorin(h), 0.01)
        big.append(kpm.create(h, a, b, precision=kpm.PREC_FP32, chunk_height=32))
    h3 = ham.ti_hamiltonian(6, 6, 6, gamma=2.0, seed=23)
    a3, b3 = kpm.scale_from_bounds(*kpm.gershgorin(h3), 0.01)
    with kpm.Batch(big, [48, 32], [32, 32], [5, 6]) as batch, \
            kpm.create(h3, a3, b3, precision=kpm.PREC_FP32, chunk_height=8) as small:
        assert batch.info()["staged_classes"] == 1
        batch.launch()
        first = [batch.eta(0), batch.eta(1)]
        ls, lb = small.get_launch(32), big[0].get_launch(32)
        assert ls["stages"] >= 1 and lb["stages"] >= 1
        assert (ls["lanes_per_row"], ls["cols_per_lane"]) == (lb["lanes_per_row"],
                                                               lb["cols_per_lane"])
        small.moments(16, 32, 7)  # plans and runs the smaller layout
        batch.launch()
        np.testing.assert_array_equal(batch.eta(0), first[0])
        np.testing.assert_array_equal(batch.eta(1), first[1])
        small.check_device_error()
    for c in big:
        c.close()
