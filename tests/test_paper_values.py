"""The build against numbers the paper prints (tests/golden/paper_printed_values.txt, each
with its passage): stencil shape and level count, network widths and depth, the parameter
count the paper rounds to 1.4 million, and the Lorenz-Mie table's mean cosine, which the
paper's HG data set matches with g = 0.857 (our droplet distribution is a reading, so it is
held to within 0.01)."""
import math
import os

from paper_1709_05418_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "paper_printed_values.txt")


def printed():
    out = {}
    for line in open(GOLDEN):
        line = line.split("#", 1)[0].strip()
        if line:
            name, *vals = line.split()
            out[name] = [float(v) for v in vals]
    return out


def test_network_shape_matches_the_paper(orc):
    v = printed()
    nx, ny, nz = (int(a) for a in v["stencil_points"])
    assert orc.DIN == nx * ny * nz + 1 == orc.stencil_din(5)
    assert orc.K == int(v["stencil_levels"][0]) and W.H == int(v["hidden_width"][0])
    shapes = W.param_shapes()
    weights = [n for n, s, fan in shapes if fan]
    # V^1, (V^k, W1^k) for k >= 2 feed one layer; W2^k the second; T1..T3 the tail
    layers = sum(1 for n in weights if n.startswith(("V", "W2", "T")))
    assert layers == int(v["network_layers"][0])
    about = v["parameters_about"][0]
    assert abs(W.param_count() - about) <= 0.1 * about
    assert list(W.SHALLOW_WIDE) == [int(a) for a in v["shallow_wide"]]


def test_lorenz_mie_mean_cosine_matches_the_paper(orc):
    p, _, ce = orc.lm_table()
    dom = 2.0 * math.pi * (ce[:-1] - ce[1:])
    g = float((p * dom * 0.5 * (ce[:-1] + ce[1:])).sum())
    assert abs(g - printed()["lm_mean_cosine"][0]) < 0.01, g


def test_record_rules_match_the_paper():
    import inspect

    from paper_1709_05418_gb300 import train
    v = printed()
    assert inspect.signature(train.records).parameters["rel_ci"].default == v["label_ci"][0]
    assert inspect.signature(train.split).parameters["train_frac"].default == v["train_split"][0]
