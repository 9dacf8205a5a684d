"""The serving loop's HBM arena (first-fit, 256-byte blocks, merging on free)
driven through a small C++ program against a brute-force model of 256-byte
units: every allocation lands where first-fit over the model's free map says,
blocks never overlap, and freeing everything leaves one block of the full size."""
import os
import random
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_1906_12085_gb300", "csrc")
UNIT = 256


@pytest.fixture(scope="module")
def driver(tmp_path_factory):
    exe = str(tmp_path_factory.mktemp("arena") / "arena_driver")
    subprocess.run(["g++", "-std=c++17", "-O1", "-I", CSRC, os.path.join(HERE, "native", "arena_driver.cpp"),
                    "-o", exe], check=True)
    return exe


def run(exe, script):
    out = subprocess.run([exe], input="\n".join(script) + "\n", capture_output=True, text=True, check=True)
    return out.stdout.split("\n")


def first_fit(free_units, n):
    """Lowest unit index starting n consecutive free units, or None."""
    run_start, run_len = None, 0
    for i, f in enumerate(free_units):
        if f:
            if run_len == 0:
                run_start = i
            run_len += 1
            if run_len == n:
                return run_start
        else:
            run_len = 0
    return None


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_arena_matches_first_fit_model(driver, seed):
    rng = random.Random(seed)
    size_units = 400
    free = [True] * size_units
    live = []       # (off, bytes)
    script = [f"i {size_units * UNIT + 100}"]  # the tail below one unit is unusable
    expect = [f"I {size_units * UNIT}"]
    for _ in range(600):
        if live and rng.random() < 0.45:
            off, nb = live.pop(rng.randrange(len(live)))
            script.append(f"r {off} {nb}")
            expect.append("R")
            u = -(-nb // UNIT)
            for j in range(off // UNIT, off // UNIT + u):
                free[j] = True
        else:
            nb = rng.choice([1, 255, 256, 257, 1000, 5000, 12345, 40000])
            u = -(-nb // UNIT)
            at = first_fit(free, u)
            script.append(f"a {nb}")
            if at is None:
                expect.append("F")
            else:
                expect.append(f"A {at * UNIT}")
                for j in range(at, at + u):
                    assert free[j]
                    free[j] = False
                live.append((at * UNIT, nb))
    for off, nb in live:
        script.append(f"r {off} {nb}")
        expect.append("R")
    script.append("s")
    expect.append(f"S 0 {size_units * UNIT} 1")
    got = run(driver, script)
    assert got[:len(expect)] == expect


def test_arena_exhaustion_and_merge(driver):
    got = run(driver, ["i 4096", "a 1024", "a 1024", "a 1024", "a 1024", "a 1", "r 1024 1024", "r 2048 1024",
                       "a 2048", "s", "r 0 1024", "r 1024 2048", "r 3072 1024", "s"])
    assert got[:14] == ["I 4096", "A 0", "A 1024", "A 2048", "A 3072", "F", "R", "R", "A 1024", "S 4096 0 0",
                        "R", "R", "R", "S 0 4096 1"]
