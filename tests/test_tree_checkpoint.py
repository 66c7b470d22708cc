"""Checkpoint and resume of the level-synchronous tree build (Proc. 3):
the state file on the CPU, and on the GPU a build interrupted after a level
that resumes to the same leaves and counts as an uninterrupted build and as
the one-call sra_extract_leaves."""
import json
import os

import numpy as np
import pytest

from paper_2202_02444_gb300 import workloads as wl


@pytest.fixture(scope="module")
def modules():
    from paper_2202_02444_gb300 import sra, tree
    return sra, tree


def nodes(rows):
    from paper_2202_02444_gb300 import sra
    return np.array([tuple(r) for r in rows], dtype=sra.NODE_DTYPE)


def test_state_round_trip_and_key_check(modules, tmp_path):
    sra, tree = modules
    path = str(tmp_path / "tree.ckpt")
    fr, lv = nodes([(1, 2, 3, 4), (5, 6, 7, 4)]), nodes([(0, 1, 0, 3)])
    counts = np.arange(sra.CNT_N, dtype=np.int64)
    tree.save_state(path, "problem-a", 4, fr, lv, counts)
    assert os.listdir(tmp_path) == ["tree.ckpt"]  # the temporary file was renamed away
    level, fr2, lv2, c2 = tree.load_state(path, "problem-a")
    assert level == 4 and np.array_equal(fr2, fr) and np.array_equal(lv2, lv) and np.array_equal(c2, counts)
    with pytest.raises(ValueError):
        tree.load_state(path, "problem-b")


def test_problem_key_covers_net_depth_and_options(modules):
    sra, tree = modules
    m1, m2 = wl.net_small_relu(), wl.make_mlp([32, 32], "relu", seed=1)
    o = sra.make_opts(arith="fixed")
    k = tree.problem_key(m1, 6, o, (-1, -1, -1), (1, 1, 1))
    assert k == tree.problem_key(m1, 6, sra.make_opts(arith="fixed"), (-1, -1, -1), (1, 1, 1))
    assert k != tree.problem_key(m2, 6, o, (-1, -1, -1), (1, 1, 1))
    assert k != tree.problem_key(m1, 7, o, (-1, -1, -1), (1, 1, 1))
    assert k != tree.problem_key(m1, 6, sra.make_opts(arith="truncate", K=8), (-1, -1, -1), (1, 1, 1))
    assert k != tree.problem_key(m1, 6, o, (-1, -1, -1), (1, 1, 2))


class Interrupt(Exception):
    pass


@pytest.mark.gpu
@pytest.mark.parametrize("arith,K,split,depth", [("fixed", 0, "octree", 6), ("truncate", 8, "kd", 14)])
def test_interrupted_build_resumes_to_the_same_tree(modules, tmp_path, arith, K, split, depth):
    sra, tree = modules
    mlp = wl.net_small_relu()
    net = sra.Net(mlp)
    try:
        opts = sra.make_opts(arith=arith, K=K, split=split)
        full_leaves, full_counts = tree.build_tree(net, depth, opts=opts)
        path = str(tmp_path / "tree.ckpt")

        def stop_at(level, n_frontier):
            if level == depth // 2:
                raise Interrupt()
        with pytest.raises(Interrupt):
            tree.build_tree(net, depth, opts=opts, checkpoint=path, on_level=stop_at)
        assert tree.load_state(path, tree.problem_key(mlp, depth, opts, (-1.0,) * 3, (1.0,) * 3))[0] == depth // 2
        log = str(tmp_path / "levels.jsonl")
        leaves, counts = tree.build_tree(net, depth, opts=opts, checkpoint=path, log=log)
        assert np.array_equal(leaves, full_leaves) and np.array_equal(counts, full_counts)
        # the log holds the resumed levels only, each with consistent counts
        recs = [json.loads(line) for line in open(log)]
        assert [r["level"] for r in recs] == list(range(depth // 2, depth + 1))
        for r in recs:
            assert r["positive"] + r["negative"] + r["unknown"] == r["frontier"]
        # without the convergence test every leaf comes from the last level,
        # one of the resumed ones
        assert sum(r["leaves"] for r in recs) == len(leaves)

        # the one-call tree on the device gives the same leaf set
        ref, _ = sra.extract_leaves(net, depth, opts=opts)
        ref_set = {tuple(r) for r in sra.tensor_to_nodes(ref).tolist()}
        assert ref_set == {tuple(r) for r in leaves.tolist()}
        assert int(full_counts[sra.CNT_LEAVES]) == len(full_leaves) > 0
        with pytest.raises(ValueError):  # the checkpoint belongs to this depth
            tree.build_tree(net, depth + 1, opts=opts, checkpoint=path)
    finally:
        net.close()
