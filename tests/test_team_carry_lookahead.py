"""The carry look-ahead rule of the warp-cooperative multi-limb kernel
(csrc/mp_team.cuh, Team::carry_in), as host arithmetic: with G the lanes
whose own sum carried out and P the lanes whose limbs are all ones
(exclusive), the carry into lane t is bit t of (U + V) xor U xor V for
U = (G | P) and V = G with every team's top lane cleared.  Checked here
exhaustively against ripple carry for teams of 2, 4 and 8 lanes, with
several teams packed into one 32-lane ballot (no carry may cross from one
team into the next)."""

import itertools
import random

import pytest

MASK32 = 0xFFFFFFFF


def top_lanes(T):
    return sum(1 << k for k in range(T - 1, 32, T))


def carry_in_word(T, G, P):
    top = top_lanes(T)
    U = (G | P) & ~top & MASK32
    V = G & ~top & MASK32
    return ((U + V) ^ U ^ V) & MASK32


def ripple(g, p):
    """carry into each lane of one team; lane 0 receives none"""
    c = [0] * len(g)
    for t in range(1, len(g)):
        c[t] = 1 if (g[t - 1] or (p[t - 1] and c[t - 1])) else 0
    return c


@pytest.mark.parametrize("T", [2, 4, 8])
def test_one_team_exhaustive(T):
    for G in range(1 << T):
        for P in range(1 << T):
            if G & P:
                continue        # a lane that carried out cannot be all ones
            g = [(G >> t) & 1 for t in range(T)]
            p = [(P >> t) & 1 for t in range(T)]
            K = carry_in_word(T, G, P)
            assert [(K >> t) & 1 for t in range(T)] == ripple(g, p), (T, G, P)


@pytest.mark.parametrize("T", [2, 4, 8])
def test_teams_packed_in_a_warp_do_not_interact(T):
    rng = random.Random(T)
    teams = 32 // T
    for _ in range(3000):
        G = P = 0
        want = []
        for k in range(teams):
            g = [rng.random() < 0.3 for _ in range(T)]
            p = [(not g[t]) and rng.random() < 0.5 for t in range(T)]
            for t in range(T):
                G |= int(g[t]) << (k * T + t)
                P |= int(p[t]) << (k * T + t)
            want += ripple(g, p)
        K = carry_in_word(T, G, P)
        assert [(K >> lane) & 1 for lane in range(32)] == want


def test_top_lane_masks():
    assert top_lanes(2) == 0xAAAAAAAA and top_lanes(4) == 0x88888888 and top_lanes(8) == 0x80808080
    assert top_lanes(32) == 0x80000000
