"""Batch schedules (lb_set_schedule, lb_autotune on a batch): how the work of
one step is cut into classes, strips, row blocks and grids changes the
launches, never the result.  Every schedule must give the state of the
same domains stepped one by one, bit for bit, in both g storages; the
autotuner must leave the state where it was."""
import numpy as np
import pytest

import lbinputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lbf():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import __graft_entry__

    __graft_entry__.build()
    import paper_0812_1282_gb300 as m

    return m


STEPS = 131  # a 64-step graph twice, a 2-step graph and one single step


def _specs():
    return lbinputs.batch_specs(n=10, seed=11, lo=40, hi=300)


def _plist(lbf, specs, compact):
    return [lbf.params(**lbinputs.BASE, collision="mrt", precision="fp32", compact_g=compact,
                       tau_alpha=s["tau_alpha"], tau_beta=s["tau_beta"],
                       h_bottom=lbf.lb_wetting_h(s["theta"]), step2_relax_momentum=True)
            for s in specs]


@pytest.fixture(scope="module", params=[False, True], ids=["full-g", "compact-g"])
def single_states(lbf, request):
    """Each domain stepped alone: the populations every schedule must give."""
    compact = request.param
    specs = _specs()
    plist = _plist(lbf, specs, compact)
    out = []
    for d, s in enumerate(specs):
        sim = lbf.Lattice(plist[d], s["nx"], s["ny"])
        sim.init_drop(s["R"], s["cx"], s["cy"])
        sim.step(STEPS)
        out.append(sim.populations())
        sim.close()
    return compact, out


def _schedules(lbf, compact):
    w = (lambda bx: (62 * (bx // 32) - 2) // 4 * 4) if compact else (lambda bx: bx)
    return {
        "one-class-persistent": lbf.schedule(128, 32, ctas_per_sm=4),
        "one-item-per-cta-largest-first": lbf.schedule(64, 16, ctas_per_sm=0, order=1),
        "two-classes-chained": lbf.schedule([64, 128], [16, 32], ctas_per_sm=[0, 3],
                                            max_nx=[w(64)], order=1),
        "two-classes-in-turn": lbf.schedule([64, 128], 8, ctas_per_sm=[2, 0], max_nx=[w(64)],
                                            chains=0),
        "three-classes": lbf.schedule([64, 96, 128], [32, 5, 64], ctas_per_sm=[1, 0, 2],
                                      max_nx=[100, 200], order=1),
        "empty-class": lbf.schedule([64, 128], 32, max_nx=[10]),
        # persistent launches (compact storage): each class's steps in one
        # launch, work items waiting on their neighbours' step flags
        "multistep-ladder": lbf.schedule([96, 160, 288], 32, ctas_per_sm=0,
                                         max_nx=[w(96), w(160)], order=1, persist=1),
        # split strips and row blocks of 3 and 5 rows: an item waits on two
        # row blocks on each side and on the strips beside it
        "multistep-short-blocks": lbf.schedule([64, 128], [5, 3], ctas_per_sm=[0, 1],
                                               max_nx=[w(64)], chains=0, persist=1),
        # one CTA per SM: most items wait for a CTA to come free
        "multistep-few-ctas": lbf.schedule(64, 16, ctas_per_sm=1, persist=1),
        # one- and two-row blocks in split strips: the most neighbours an item
        # can wait for (five row blocks in three strips)
        "multistep-single-rows": lbf.schedule([32, 64], [1, 2], ctas_per_sm=0, max_nx=[w(32)],
                                              order=1, persist=1),
        # over-filled: some CTAs start only when a class finishes
        "multistep-overfilled-sealed": lbf.schedule([96, 160, 288], 32, ctas_per_sm=0,
                                                    max_nx=[w(96), w(160)], order=1,
                                                    persist=1, fill_pct=150, seal_edges=1),
        # every compute-warp count 2..9, all classes on the one kernel body
        # built for any width
        "eight-class-ladder": lbf.schedule([64, 96, 128, 160, 192, 224, 256, 288], 16,
                                           ctas_per_sm=0, order=1,
                                           max_nx=[w(b) for b in (64, 96, 128, 160, 192, 224, 256)]),
        # whole-domain strips that write whole sectors (zeroed ghost columns)
        "sealed-ladder": lbf.schedule([96, 160, 288], 64, ctas_per_sm=0,
                                      max_nx=[w(96), w(160)], order=1, seal_edges=[1, 0, 1]),
    }


MULTISTEP = ("multistep-ladder", "multistep-short-blocks", "multistep-few-ctas",
             "multistep-overfilled-sealed", "multistep-single-rows")


@pytest.mark.parametrize("name", ["one-class-persistent", "one-item-per-cta-largest-first",
                                  "two-classes-chained", "two-classes-in-turn", "three-classes",
                                  "empty-class", "eight-class-ladder", "sealed-ladder",
                                  *MULTISTEP])
def test_schedule_gives_single_domain_results(lbf, single_states, name):
    compact, ref = single_states
    if (name in MULTISTEP or name in ("sealed-ladder", "eight-class-ladder")) and not compact:
        pytest.skip("persistent launches, sealing and 288-wide strips take compact storage")
    specs = _specs()
    plist = _plist(lbf, specs, compact)
    batch = lbf.Batch(plist, [s["nx"] for s in specs], [s["ny"] for s in specs])
    batch.set_schedule(_schedules(lbf, compact)[name])
    got = batch.schedule()
    assert got["n_class"] == _schedules(lbf, compact)[name].n_class
    for d, s in enumerate(specs):
        batch.init_drop(s["R"], s["cx"], s["cy"], dom=d)
    batch.step(STEPS)
    for d in range(len(specs)):
        fb, gb = batch.populations(dom=d)
        assert np.array_equal(fb, ref[d][0]) and np.array_equal(gb, ref[d][1]), (name, d)
    batch.close()


def test_autotune_keeps_state_and_picks_valid_schedule(lbf):
    specs = _specs()
    plist = _plist(lbf, specs, True)
    batch = lbf.Batch(plist, [s["nx"] for s in specs], [s["ny"] for s in specs])
    for d, s in enumerate(specs):
        batch.init_drop(s["R"], s["cx"], s["cy"], dom=d)
    batch.step(7)
    before = batch.save_state()
    bx, rows, ms = batch.autotune(reps=1)
    assert batch.save_state() == before
    sc = batch.schedule()
    assert sc["block_x"][0] == bx and sc["rows"][0] == rows and ms > 0
    assert 1 <= sc["n_class"] <= 8 and sc["order"] in (0, 1)
    # and stepping on with the chosen schedule still matches a fresh run
    batch.step(20)
    other = lbf.Batch(plist, [s["nx"] for s in specs], [s["ny"] for s in specs])
    for d, s in enumerate(specs):
        other.init_drop(s["R"], s["cx"], s["cy"], dom=d)
    other.step(27)
    assert other.save_state()[32:] == batch.save_state()[32:]
    batch.close()
    other.close()


def test_fp64_ladder_matches_single_domains(lbf):
    """FP64 (full g storage): a two-class ladder, whose classes both launch
    the one kernel body built for any width, and a single class on the body
    built for its width give each domain's single-domain state bit for bit
    (walls, 64- and 128-column strips, domains split over several strips)."""
    specs = _specs()[:6]
    plist = [lbf.params(**lbinputs.BASE, collision="mrt", precision="fp64",
                        tau_alpha=s["tau_alpha"], tau_beta=s["tau_beta"],
                        h_bottom=lbf.lb_wetting_h(s["theta"]), step2_relax_momentum=True)
             for s in specs]
    steps = 67
    ref = []
    for d, s in enumerate(specs):
        sim = lbf.Lattice(plist[d], s["nx"], s["ny"])
        sim.init_drop(s["R"], s["cx"], s["cy"])
        sim.step(steps)
        ref.append(sim.populations())
        sim.close()
    for sc in (lbf.schedule([64, 128], 16, ctas_per_sm=0, max_nx=[100], order=1),
               lbf.schedule(128, 16, ctas_per_sm=0)):
        batch = lbf.Batch(plist, [s["nx"] for s in specs], [s["ny"] for s in specs])
        batch.set_schedule(sc)
        for d, s in enumerate(specs):
            batch.init_drop(s["R"], s["cx"], s["cy"], dom=d)
        batch.step(steps)
        for d in range(len(specs)):
            fb, gb = batch.populations(dom=d)
            assert np.array_equal(fb, ref[d][0]) and np.array_equal(gb, ref[d][1]), (sc.n_class, d)
        batch.close()


def test_schedule_validation(lbf):
    specs = _specs()[:3]
    plist = _plist(lbf, specs, True)
    batch = lbf.Batch(plist, [s["nx"] for s in specs], [s["ny"] for s in specs])
    bad = [lbf.schedule(48, 32),                                  # not a multiple of 32
           lbf.schedule(128, 0),                                  # no rows
           lbf.schedule(128, 32, ctas_per_sm=33),                 # too many CTAs per SM
           lbf.schedule([64, 128, 128], 32, max_nx=[200, 100]),   # limits not increasing
           lbf.schedule(128, 32, order=2),
           lbf.schedule(128, 32, persist=2),
           lbf.schedule(128, 32, persist=1, fill_pct=401),
           lbf.schedule(128, 32, seal_edges=2)]
    for sc in bad:
        with pytest.raises(lbf.LBError) as e:
            batch.set_schedule(sc)
        assert e.value.code == lbf.LB_ERR_INVALID_ARG
    sc = lbf.Schedule()
    sc.n_class = 9
    with pytest.raises(lbf.LBError):
        batch.set_schedule(sc)
    batch.close()
    # persistent launches are built for compact FP32 storage only
    full = lbf.Batch(_plist(lbf, specs, False), [s["nx"] for s in specs],
                     [s["ny"] for s in specs])
    with pytest.raises(lbf.LBError) as e:
        full.set_schedule(lbf.schedule(128, 32, persist=1))
    assert e.value.code == lbf.LB_ERR_INVALID_ARG
    full.close()


@pytest.mark.parametrize("compact,persist", [(False, 0), (True, 0), (True, 1)],
                         ids=["full-g", "compact-g", "compact-g-multistep"])
def test_switching_schedules_midrun_matches_a_fixed_schedule(lbf, compact, persist):
    """Strips that cover a whole domain wrap in shared memory and leave the
    ghost columns alone (compact storage); a later schedule that splits the
    same domains into several strips must still see correct ghost columns.
    Whole -> split -> whole, with a checkpoint in between, against a run on
    one split schedule throughout (the whole-strip schedule also as
    persistent multi-step launches)."""
    specs = _specs()
    plist = _plist(lbf, specs, compact)
    nxs, nys = [s["nx"] for s in specs], [s["ny"] for s in specs]
    whole = lbf.schedule(256, 16, ctas_per_sm=0, persist=persist,  # every domain one strip
                         seal_edges=persist)
    split = lbf.schedule(32, 7, ctas_per_sm=2, order=1)  # strips of 60 (compact) / 32 columns

    def init(b):
        for d, s in enumerate(specs):
            b.init_drop(s["R"], s["cx"], s["cy"], dom=d)

    ref = lbf.Batch(plist, nxs, nys)
    ref.set_schedule(split)
    init(ref)
    ref.step(90)
    b = lbf.Batch(plist, nxs, nys)
    b.set_schedule(whole)
    init(b)
    b.step(30)
    b.set_schedule(split)
    b.step(30)
    blob = b.save_state()
    b.set_schedule(whole)
    b.step(17)
    b.load_state(blob)
    b.set_schedule(split)
    b.step(30)
    for d in range(len(specs)):
        fr, gr = ref.populations(dom=d)
        fb, gb = b.populations(dom=d)
        assert np.array_equal(fr, fb) and np.array_equal(gr, gb), d
    assert ref.save_state()[32:] == b.save_state()[32:]
    ref.close()
    b.close()
