"""Model files (Sec. 3.1): the bmdp-tool and PRISM explicit readers and writers
of the C ABI. Host-only calls: these tests need no GPU.

The fixtures in tests/golden/ are the Sec. 3.1 model written by hand in both
formats (SOURCES.txt there); they must read back as the same CSC arrays as the
JSON fixture, and the query in the .pctl file as the Sec. 3.2 query."""
import os
from fractions import Fraction as Fr

import numpy as np
import pytest

import oracle
import paper_2401_04068_gb300 as g
from exact_lp import columns_from_csc, exact_value_iteration
from workloads import random_imdp

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2401_04068_gb300 import build
    build.build()
    g.load()


def _same_arrays(f, m):
    np.testing.assert_array_equal(f.stateptr, m["stateptr"] if isinstance(m, dict) else m.stateptr)
    for name in ("colptr", "rowval", "lower", "upper"):
        a = getattr(f, name)
        b = m[name] if isinstance(m, dict) else getattr(m, name)
        np.testing.assert_array_equal(a, b, err_msg=name)


def _status(exc_info):
    return exc_info.value.status


# --------------------------------------------------------------------------- the hand-written fixtures

def test_bmdp_fixture_is_the_worked_example(worked_example):
    f = g.imdp_read_bmdp_tool(os.path.join(GOLDEN, "worked_example.bmdp"))
    assert f.n_states == 3
    _same_arrays(f, worked_example)
    assert list(f.action) == [0, 1, 0, 1, 0]
    s = f.spec
    assert list(s["reach"]) == [2] and s["property"] == g.IMDP_REACH
    # the format has no horizon or modes: the documented defaults
    assert s["horizon"] == 0 and not s["infinite_time"] and s["pessimistic"] and s["maximize"]


def test_prism_fixture_is_the_worked_example_and_its_query(worked_example):
    f = g.imdp_read_prism(os.path.join(GOLDEN, "worked_example"))
    _same_arrays(f, worked_example)
    assert list(f.action) == [0, 1, 0, 1, 0]
    s = f.spec
    assert s["property"] == g.IMDP_REACH and list(s["reach"]) == [2] and len(s["avoid"]) == 0
    assert s["horizon"] == 100 and not s["infinite_time"] and s["pessimistic"] and s["maximize"]


def _exact_columns_from_bmdp_text(path):
    """Bounds of the bmdp fixture as exact decimals, straight from the text."""
    lines = open(path).read().split()
    n, _, nt = int(lines[0]), int(lines[1]), int(lines[2])
    rest = lines[3 + nt:]
    ent = sorted((int(rest[i]), int(rest[i + 1]), int(rest[i + 2]), Fr(rest[i + 3]), Fr(rest[i + 4]))
                 for i in range(0, len(rest), 5))
    return n, ent


def test_bmdp_fixture_values_match_exact_value_iteration():
    # file text -> exact rationals -> Eq. 2 by LP vertex enumeration, against the
    # oracle run on what the reader returned
    path = os.path.join(GOLDEN, "worked_example.bmdp")
    f = g.imdp_read_bmdp_tool(path)
    n, ent = _exact_columns_from_bmdp_text(path)
    exact = [(lo, up) for (_, _, _, lo, up) in ent]
    cols = columns_from_csc(f.colptr, f.rowval, f.lower, f.upper, exact_values=exact)
    hist, _ = exact_value_iteration(n, cols, f.stateptr, list(f.spec["reach"]), 5, True, True)
    assert hist[1] == [Fr(1, 5), Fr(2, 5), Fr(1)]
    assert hist[2] == [Fr(21, 50), Fr(29, 50), Fr(1)]
    m = oracle.OracleIMDP(f.n_states, f.stateptr, f.colptr, f.rowval, f.lower, f.upper)
    for k in (1, 2, 5):
        st, V, kk, _, _ = oracle.value_iteration(m, oracle.OracleSpec(horizon=k, reach=list(f.spec["reach"])))
        assert st == "ok" and kk == k
        np.testing.assert_allclose(V, [float(x) for x in hist[k]], rtol=0, atol=1e-15)


# --------------------------------------------------------------------------- round trips

@pytest.mark.parametrize("seed", range(4))
def test_bmdp_round_trip_is_bitwise(tmp_path, seed):
    m = random_imdp(40 + 17 * seed, max_actions=4, seed=300 + seed)
    p = tmp_path / "m.bmdp"
    g.imdp_write_bmdp_tool(p, m, m.goal)
    f = g.imdp_read_bmdp_tool(p)
    _same_arrays(f, m)
    sp = np.asarray(m.stateptr)
    assert list(f.action) == [j - sp[s] for s in range(m.n_states) for j in range(sp[s], sp[s + 1])]
    assert list(f.spec["reach"]) == sorted(set(np.asarray(m.goal).tolist()))


SPECS = [
    dict(horizon=7, pessimistic=True, maximize=True),
    dict(horizon=0, pessimistic=False, maximize=False),
    dict(infinite_time=True, pessimistic=True, maximize=False),
    dict(property=g.IMDP_REACH_AVOID, horizon=12, pessimistic=False, maximize=True),
    dict(property=g.IMDP_REACH_AVOID, infinite_time=True, pessimistic=True, maximize=True),
]


@pytest.mark.parametrize("i", range(len(SPECS)))
def test_prism_round_trip_is_bitwise(tmp_path, i):
    m = random_imdp(55, max_actions=3, seed=400 + i)
    kw = dict(SPECS[i])
    kw["reach"] = m.goal
    if kw.get("property") == g.IMDP_REACH_AVOID:
        goal = set(np.asarray(m.goal).tolist())
        kw["avoid"] = [s for s in range(0, m.n_states, 5) if s not in goal][:6]
    g.imdp_write_prism(tmp_path / "m", m, **kw)
    f = g.imdp_read_prism(tmp_path / "m")
    _same_arrays(f, m)
    s = f.spec
    assert s["property"] == kw.get("property", g.IMDP_REACH)
    assert s["infinite_time"] == kw.get("infinite_time", False)
    if not s["infinite_time"]:
        assert s["horizon"] == kw["horizon"]
    assert s["pessimistic"] == kw["pessimistic"] and s["maximize"] == kw["maximize"]
    assert list(s["reach"]) == sorted(set(np.asarray(m.goal).tolist()))
    assert list(s["avoid"]) == sorted(kw.get("avoid", []))


def test_bmdp_writer_output_read_independently(tmp_path):
    # the written text against the documented layout, parsed here in Python
    m = random_imdp(30, max_actions=3, seed=500)
    p = tmp_path / "m.bmdp"
    g.imdp_write_bmdp_tool(p, m, [3, 1])
    lines = open(p).read().splitlines()
    sp, cp = np.asarray(m.stateptr), np.asarray(m.colptr)
    assert int(lines[0]) == m.n_states
    assert int(lines[1]) == int(np.diff(sp).max())
    assert int(lines[2]) == 2 and [int(x) for x in lines[3:5]] == [3, 1]
    rows = [ln.split() for ln in lines[5:]]
    assert len(rows) == len(m.rowval)
    e = 0
    for s in range(m.n_states):
        for j in range(sp[s], sp[s + 1]):
            for k in range(cp[j], cp[j + 1]):
                src, act, dst, lo, up = rows[e]
                assert (int(src), int(act), int(dst)) == (s, j - sp[s], int(m.rowval[k]))
                assert float(lo) == m.lower[k] and float(up) == m.upper[k]
                e += 1


def test_prism_writer_output_read_independently(tmp_path):
    m = random_imdp(20, max_actions=2, seed=501)
    g.imdp_write_prism(tmp_path / "m", m, property=g.IMDP_REACH_AVOID, horizon=9, pessimistic=True,
                       maximize=False, reach=[4], avoid=[0, 7])
    sta = open(tmp_path / "m.sta").read().splitlines()
    assert sta[0].startswith("(") and len(sta) == m.n_states + 1
    lab = open(tmp_path / "m.lab").read().splitlines()
    assert '2="reach"' in lab[0] and '3="avoid"' in lab[0]
    labels = {int(l.split(":")[0]): l.split(":")[1].split() for l in lab[1:]}
    assert labels[4] == ["2"] and "3" in labels[0] and "0" in labels[0] and labels[7] == ["3"]
    tra = open(tmp_path / "m.tra").read().splitlines()
    assert [int(x) for x in tra[0].split()] == [m.n_states, len(m.colptr) - 1, len(m.rowval)]
    first = tra[1].split()
    lo, up = first[3].strip("[]").split(",")
    assert float(lo) == m.lower[0] and float(up) == m.upper[0]
    assert open(tmp_path / "m.pctl").read().strip() == 'Pminmin=? [ !"avoid" U<=9 "reach" ]'


# --------------------------------------------------------------------------- structure the readers supply

def test_state_without_transitions_becomes_absorbing(tmp_path):
    p = tmp_path / "a.bmdp"
    p.write_text("4\n1\n1\n3\n0 0 1 0.5 0.5\n0 0 3 0.5 0.5\n1 0 3 1 1\n3 0 3 1 1\n")
    f = g.imdp_read_bmdp_tool(p)
    assert list(f.stateptr) == [0, 1, 2, 3, 4]
    # state 2 has no line: one column holding its self-loop [1, 1], action -1
    assert list(f.action) == [0, 0, -1, 0]
    j = f.stateptr[2]
    assert list(f.rowval[f.colptr[j]:f.colptr[j + 1]]) == [2]
    assert f.lower[f.colptr[j]] == 1.0 and f.upper[f.colptr[j]] == 1.0


def test_bmdp_actions_with_gaps_keep_their_indices(tmp_path):
    p = tmp_path / "g.bmdp"
    p.write_text("2\n3\n0\n0 2 1 1 1\n0 0 0 1 1\n1 1 1 1 1\n")
    f = g.imdp_read_bmdp_tool(p)
    assert list(f.stateptr) == [0, 2, 3] and list(f.action) == [0, 2, 1]


@pytest.mark.parametrize("prop,expect", [
    ('Pmaxmin=? [ F<=10 "goal" ]', dict(property=0, infinite_time=False, horizon=10, pessimistic=True,
                                        maximize=True)),
    ('Pminmax=?[F "goal"]', dict(property=0, infinite_time=True, pessimistic=False, maximize=False)),
    ('Pmaxmax=? [ !"bad" U<=5 "goal" ]', dict(property=1, infinite_time=False, horizon=5, pessimistic=False,
                                              maximize=True)),
    ('Pminmin=? [ (!"bad") U "goal" ]', dict(property=1, infinite_time=True, pessimistic=True, maximize=False)),
    ('Pmax=? [ F<=3 "goal" ]', dict(property=0, horizon=3, pessimistic=True, maximize=True)),
])
def test_prism_property_forms(tmp_path, prop, expect):
    (tmp_path / "p.sta").write_text("(x)\n0:(0)\n1:(1)\n")
    (tmp_path / "p.lab").write_text('0="init" 1="goal" 2="bad"\n0: 0 2\n1: 1\n')
    (tmp_path / "p.tra").write_text("2 2 3\n0 0 0 [0.2,0.6]\n0 0 1 [0.4,0.8]\n1 0 1 1\n")
    (tmp_path / "p.pctl").write_text(prop + "\n")
    f = g.imdp_read_prism(tmp_path / "p")
    for k, v in expect.items():
        assert f.spec[k] == v, (k, f.spec[k], v)
    assert list(f.spec["reach"]) == [1]
    assert list(f.spec["avoid"]) == ([0] if expect["property"] == 1 else [])
    if expect.get("infinite_time"):
        assert f.spec["eps"] == 1e-6


# --------------------------------------------------------------------------- errors

BMDP_BAD = [
    ("0\n1\n0\n", "number of states"),
    ("2\n1\n1\n5\n", "terminal state"),
    ("2\n1\n0\n0 0 2 0.5 0.5\n", "out of range"),
    ("2\n1\n0\n0 1 1 0.5 0.5\n", "action index"),
    ("2\n1\n0\n0 0 1 0.5 0.5\n0 0 1 0.5 0.5\n", "duplicate"),
    ("2\n1\n0\n0 0 1 0.5\n1 0 1 1 1\n", "expected: source"),
    ("2\n1\n0\n0 0 1 x 0.5\n", "expected: source"),
    ("2\n1\n0\n0 0 1 nan 0.5\n", "finite"),
]


@pytest.mark.parametrize("text,msg", BMDP_BAD)
def test_bmdp_rejects_malformed_files(tmp_path, text, msg):
    p = tmp_path / "bad.bmdp"
    p.write_text(text)
    with pytest.raises(g.ImdpError) as e:
        g.imdp_read_bmdp_tool(p)
    assert _status(e) == g.IMDP_EINVAL
    assert msg in str(e.value) and "bad.bmdp:" in str(e.value)


def _prism(tmp_path, sta="(x)\n0:(0)\n1:(1)\n", lab='0="init" 1="goal"\n1: 1\n',
           tra="2 2 3\n0 0 0 [0.2,0.6]\n0 0 1 [0.4,0.8]\n1 0 1 1\n", pctl='Pmaxmin=? [ F<=4 "goal" ]\n'):
    for ext, text in (("sta", sta), ("lab", lab), ("tra", tra), ("pctl", pctl)):
        (tmp_path / f"p.{ext}").write_text(text)
    return tmp_path / "p"


PRISM_BAD = [
    (dict(tra="2 2 4\n0 0 0 [0.2,0.6]\n0 0 1 [0.4,0.8]\n1 0 1 1\n"), "transitions"),
    (dict(tra="2 3 3\n0 0 0 [0.2,0.6]\n0 0 1 [0.4,0.8]\n1 0 1 1\n"), "choices"),
    (dict(tra="2 2 3\n0 1 0 [0.2,0.6]\n0 1 1 [0.4,0.8]\n1 0 1 1\n"), "no choice 0"),
    (dict(tra="2 2 3\n0 0 0 [0.2,0.6\n0 0 1 [0.4,0.8]\n1 0 1 1\n"), "expected: source"),
    (dict(sta="(x)\n0:(0)\n"), "lists 1 states"),
    (dict(lab='0="init" 1="goal"\n1: 4\n'), "not declared"),
    (dict(pctl='Pmaxmin=? [ F<=4 "target" ]\n'), "not in .lab"),
    (dict(pctl='R{"cost"}max=? [ F "goal" ]\n'), "reward"),
    (dict(pctl='Pmaxmin=? [ G "goal" ]\n'), "expected F"),
    (dict(pctl='Pmaxmin=? [ F<=x "goal" ]\n'), "<=K"),
]


@pytest.mark.parametrize("kw,msg", PRISM_BAD)
def test_prism_rejects_malformed_files(tmp_path, kw, msg):
    stem = _prism(tmp_path, **kw)
    with pytest.raises(g.ImdpError) as e:
        g.imdp_read_prism(stem)
    assert _status(e) == g.IMDP_EINVAL
    assert msg in str(e.value)


def test_missing_files_and_unwritable_paths_are_io_errors(tmp_path):
    with pytest.raises(g.ImdpError) as e:
        g.imdp_read_bmdp_tool(tmp_path / "none.bmdp")
    assert _status(e) == g.IMDP_EIO
    stem = _prism(tmp_path)
    os.remove(str(stem) + ".lab")
    with pytest.raises(g.ImdpError) as e:
        g.imdp_read_prism(stem)
    assert _status(e) == g.IMDP_EIO and ".lab" in str(e.value)
    m = random_imdp(5, seed=502)
    with pytest.raises(g.ImdpError) as e:
        g.imdp_write_bmdp_tool(tmp_path / "no_such_dir" / "m.bmdp", m, [0])
    assert _status(e) == g.IMDP_EIO


def test_writers_reject_what_the_formats_cannot_hold(tmp_path):
    m = random_imdp(6, seed=503)
    with pytest.raises(g.ImdpError) as e:
        g.imdp_write_prism(tmp_path / "r", m, property=g.IMDP_REWARD, reward=np.ones(6), discount=0.9)
    assert _status(e) == g.IMDP_EINVAL and "reachability" in str(e.value)
    # a column without transitions cannot be written (nor is it a feasible interval column)
    cp = np.asarray(m.colptr).copy()

    class Empty:
        n_states = m.n_states
        stateptr = m.stateptr
        colptr = np.concatenate([[0], cp[:-1]]).astype(np.int32)  # column 0 empty, last entries dropped
        rowval = np.asarray(m.rowval)[:cp[-2]]
        lower = np.asarray(m.lower)[:cp[-2]]
        upper = np.asarray(m.upper)[:cp[-2]]
    with pytest.raises(g.ImdpError) as e:
        g.imdp_write_bmdp_tool(tmp_path / "e.bmdp", Empty, [0])
    assert _status(e) == g.IMDP_EINVAL and "at least one transition" in str(e.value)
    with pytest.raises(g.ImdpError) as e:
        g.imdp_write_bmdp_tool(tmp_path / "t.bmdp", m, [6])
    assert _status(e) == g.IMDP_EINVAL


def test_mutated_fixtures_are_read_or_rejected(tmp_path):
    # byte-level mutations of the hand-written files: every one is either read
    # into arrays that satisfy the CSC structure or rejected with a status
    # (never a crash), and error text is always returned
    import random
    rng = random.Random(7)
    exts = ["bmdp", "sta", "lab", "tra", "pctl"]
    base = {e: open(os.path.join(GOLDEN, "worked_example." + e), "rb").read() for e in exts}
    alphabet = b" \t\n\r0123456789.-+e[],:=\"!()FUPRmaxin<>?/" + bytes([0, 128, 255])
    accepted = 0
    for _ in range(600):
        which = rng.choice(exts)
        for e in exts:
            b = bytearray(base[e])
            if e == which:
                for _ in range(rng.randint(1, 5)):
                    op = rng.randrange(3)
                    if op == 0 and b:
                        del b[rng.randrange(len(b))]
                    elif op == 1:
                        b.insert(rng.randrange(len(b) + 1), rng.choice(alphabet))
                    elif b:
                        b[rng.randrange(len(b))] = rng.choice(alphabet)
            (tmp_path / f"f.{e}").write_bytes(bytes(b))
        try:
            f = g.imdp_read_bmdp_tool(tmp_path / "f.bmdp") if which == "bmdp" else g.imdp_read_prism(tmp_path / "f")
        except g.ImdpError as e:
            assert e.status in (g.IMDP_EINVAL, g.IMDP_ENOMEM) and str(e)
            continue
        accepted += 1
        sp, cp, rv = f.stateptr, f.colptr, f.rowval
        assert sp[0] == 0 and np.all(np.diff(sp) >= 1) and sp[-1] == len(cp) - 1
        assert cp[0] == 0 and np.all(np.diff(cp) >= 1) and cp[-1] == len(rv)
        assert np.all((rv >= 0) & (rv < f.n_states))
        assert all(np.all(np.diff(rv[cp[j]:cp[j + 1]]) > 0) for j in range(len(cp) - 1))
        assert np.all(np.isfinite(f.lower)) and np.all(np.isfinite(f.upper))
    assert 0 < accepted < 600


def test_large_files_are_read_in_parts_in_file_order(tmp_path):
    # files above 1 MB are parsed on several host threads: arrays, order and the
    # line number of an error deep in the file must not depend on that
    import random
    from workloads import banded_imdp
    m = banded_imdp(3000, 2, 3000 * 2 * 20 + 1, seed=95)
    p = tmp_path / "big.bmdp"
    g.imdp_write_bmdp_tool(p, m, m.goal)
    assert os.path.getsize(p) > (4 << 20)
    _same_arrays(g.imdp_read_bmdp_tool(p), m)
    lines = open(p).read().splitlines()
    header, body = lines[:3 + len(m.goal)], lines[3 + len(m.goal):]
    random.Random(1).shuffle(body)  # any line order reads back the same
    p.write_text("\n".join(header + body) + "\n")
    _same_arrays(g.imdp_read_bmdp_tool(p), m)
    bad = len(lines) - 1234  # 0-based index of a line near the end
    lines[bad] = "0 0 x 0.5 0.5"
    p.write_text("\n".join(lines) + "\n")
    with pytest.raises(g.ImdpError) as e:
        g.imdp_read_bmdp_tool(p)
    assert f"big.bmdp:{bad + 1}:" in str(e.value)

    g.imdp_write_prism(tmp_path / "big", m, horizon=50, reach=m.goal)
    _same_arrays(g.imdp_read_prism(tmp_path / "big"), m)
    tra = open(tmp_path / "big.tra").read().splitlines()
    bad = len(tra) // 2 + 7
    tra[bad] = tra[bad].replace("[", "(")
    (tmp_path / "big.tra").write_text("\n".join(tra) + "\n")
    with pytest.raises(g.ImdpError) as e:
        g.imdp_read_prism(tmp_path / "big")
    assert f"big.tra:{bad + 1}:" in str(e.value)
