"""Host logic of the leaf-size autotuner: the table lookup by size class."""
from paper_0908_0673_gb300 import bem, tune


def test_choose_by_size_class():
    table = {"laplace-mixed": [{"max_elems": 4000, "leaf_size": 32}, {"max_elems": 60000, "leaf_size": 64},
                               {"max_elems": 15000, "leaf_size": 48}]}
    pick = lambda n: tune.choose(n, bem.BEM_LAPLACE, bem.BEM_MIXED, table)["leaf_size"]
    assert pick(1000) == 32 and pick(4000) == 32
    assert pick(4001) == 48 and pick(15000) == 48
    assert pick(30000) == 64 and pick(10 ** 6) == 64       # beyond the last class: the last class's choice
    assert tune.choose(5000, bem.BEM_HELMHOLTZ, bem.BEM_F64, table)["leaf_size"] == tune.DEFAULT_LEAF
    prm = tune.choose(5000, bem.BEM_LAPLACE, bem.BEM_MIXED, table)
    assert prm["p"] == 10 and prm["eta"] == 2.0 and prm["precision"] == bem.BEM_MIXED


def test_representative_meshes_grow_with_class():
    sizes = [tune._representative(hi).n_elems for hi in tune.CLASSES[:3]]
    assert sizes == sorted(sizes)
    lo = 1000
    for hi, n in zip(tune.CLASSES, sizes):
        assert lo * 0.7 <= n <= hi * 1.3
        lo = hi
