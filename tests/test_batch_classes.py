"""The classes a batch is cut into (mcpd_batch_classes, the rule mcpd_batch_create applies), on the
host: automatic classes group coupled instances by uniform degree and cut every group by pair
state into the batch's class count; a fixed count cuts all instances by pair state alone."""
import numpy as np
import pytest

import synth
from paper_2608_30239_gb300 import mcpd


def _degree(inst):
    d = np.diff(inst.clone_ptr)
    return int(d[0]) if np.all(d == d[0]) else 0


def _wpp(inst):
    # words per pair column: the clone bits, then one count byte per pool and the padding pool
    return (inst.n + 31) // 32 + (inst.m + 1 + 3) // 4


def _bench_batch():
    insts = synth.batched_configs(512, seed=11)
    ps = [dict(slots=1024, horizon=20 * i.n, seed=5000 + k, instance_id=k, meeting_cap=20 * i.n)
          for k, i in enumerate(insts)]
    return insts, ps


def test_automatic_classes_of_the_bench_batch():
    """512 uneven instances (degrees 4 to 8), 1024 slots each on 152 SMs: four classes for each
    degree, every class of one degree, the classes of a degree numbered together, largest pair
    state first, and every class holding an instance."""
    insts, ps = _bench_batch()
    cls, n = mcpd.batch_classes(insts, ps)
    deg = np.array([_degree(i) for i in insts])
    wpp = np.array([_wpp(i) for i in insts])
    assert n == 20 and sorted(set(cls.tolist())) == list(range(20))
    groups = [sorted(set(deg[cls == c].tolist())) for c in range(n)]
    assert all(len(g) == 1 for g in groups)
    assert [g[0] for g in groups] == [d for d in (4, 5, 6, 7, 8) for _ in range(4)]
    for c in range(n - 1):
        if groups[c] == groups[c + 1]:
            assert wpp[cls == c].min() >= wpp[cls == c + 1].max()


def test_fixed_class_count_cuts_by_size_only():
    """A fixed class count ignores the degrees: classes of decreasing pair state, of about equal
    work (slots x slot length), mixing degrees."""
    insts, ps = _bench_batch()
    cls, n = mcpd.batch_classes(insts, ps, classes=3)
    wpp = np.array([_wpp(i) for i in insts])
    work = np.array([1024.0 * 20 * i.n for i in insts])
    assert n == 3
    for c in range(n - 1):
        assert wpp[cls == c].min() >= wpp[cls == c + 1].max()
    shares = np.array([work[cls == c].sum() for c in range(n)]) / work.sum()
    assert np.all(np.abs(shares - 1 / 3) < 0.05)
    assert all(len(set(_degree(i) for i, c in zip(insts, cls) if c == k)) > 1 for k in range(n))


def test_degree_groups_of_a_small_batch():
    """Few slots (under one launch): one class per degree group, the mixed-degree instance in the
    generic group (numbered first), instances of one degree together."""
    insts = [synth.make_instance(150 + 90 * i, 14 + i, d, 2, 0.05, 0.12, 2 / (150 + 90 * i), 970 + i, 980 + i)
             for i, d in enumerate([4, 7, 4, 5, 7, 4])]
    insts.append(synth.make_mixed_instance(260, 21, 2, 7, 3, 0.08, 0.18, 3 / 260, 990, 991))
    ps = [dict(slots=300, k=3, ell=40, horizon=160, seed=1 + i, instance_id=i) for i in range(len(insts))]
    cls, n = mcpd.batch_classes(insts, ps)
    assert n == 4
    assert cls[6] == 0                                        # the mixed-degree instance
    assert cls[0] == cls[2] == cls[5] and cls[1] == cls[4]
    assert len({cls[0], cls[1], cls[3], cls[6]}) == 4
    assert [cls[3] > cls[0], cls[1] > cls[3]] == [True, True]   # degree 4, then 5, then 7


def test_more_multiprocessors_fewer_classes():
    """The automatic class count is the number of whole launches the slots fill (at most four):
    on a GPU with 1000 multiprocessors the bench batch fills none, so each degree keeps one class."""
    insts, ps = _bench_batch()
    cls, n = mcpd.batch_classes(insts, ps, sm_count=1000)
    assert n == 5
    assert all(len({_degree(i) for i, c in zip(insts, cls) if c == k}) == 1 for k in range(n))


def test_uncoupled_batches_are_not_grouped_by_degree():
    insts, ps = _bench_batch()
    ps = [dict(slots=1024, coupled=False, burn=10, length=100, horizon=20 * i.n, seed=5000 + k, instance_id=k)
          for k, i in enumerate(insts)]
    cls, n = mcpd.batch_classes(insts, ps)
    assert n == 4
    assert all(len({_degree(i) for i, c in zip(insts, cls) if c == k}) > 1 for k in range(n))


def test_invalid_inputs_are_refused():
    insts, ps = _bench_batch()
    with pytest.raises(mcpd.McpdError):
        mcpd.batch_classes(insts[:3], ps[:3], sm_count=0)
    with pytest.raises(mcpd.McpdError):
        mcpd.batch_classes(insts[:3], ps[:3], classes=9)
