"""Host model of the split-BF16 contraction's slot protocol (no device).

Producer teams take chunks i = t, t + T, t + 2T, ... (T teams); chunk i goes to A/B slot
s = i mod S (S slots).  Before writing a slot, a team waits for the MMAs of the slot's previous
use (chunk i - S) through a parity wait on the slot's barrier: the wait passes when the number c
of completed phases has the parity of u = i // S, so it is unambiguous only while c is u - 1 or u
when the wait starts.  If c could still be u - 2 (the MMAs of chunk i - 2S not complete), the
parity would match too early and the team would overwrite a slot the tensor core still reads.
The issuer consumes chunks in order and their MMAs complete in order.

The model explores random interleavings of the teams, the issuer and the MMA completions and
checks that every wait starts with c in {u - 1, u} when T <= S (the rule the kernel enforces by
capping its teams at its slots), and finds a schedule that breaks it when T > S.
"""
import random

import pytest


def run(T, S, nch, rng):
    """One random schedule; returns the first aliasing wait (chunk, completed phases, use) or None."""
    team_next = list(range(T))               # next chunk of each team
    team_state = ["wait"] * T                # "wait": about to wait on the slot; "write": writing it
    produced = [False] * nch
    completed = [0] * S                      # completed phases of each slot's barrier
    issued = 0                               # chunks whose MMAs the issuer has started
    done = 0                                 # chunks whose MMAs have completed (in order)
    while done < nch:
        moves = []
        for t in range(T):
            i = team_next[t]
            if i >= nch:
                continue
            u = i // S
            if team_state[t] == "wait":
                if u == 0 or completed[i % S] % 2 == u % 2:  # the parity wait passes
                    moves.append(("pass", t))
            else:
                moves.append(("produce", t))
        if issued < nch and produced[issued]:
            moves.append(("issue", None))
        if done < issued:
            moves.append(("complete", None))
        assert moves, "no move: the protocol stalls"
        kind, t = rng.choice(moves)
        if kind == "pass":
            i = team_next[t]
            u, c = i // S, completed[i % S]
            if u > 0 and c != u:                 # passed without the MMAs of chunk i - S complete
                return i, c, u
            team_state[t] = "write"
        elif kind == "produce":
            produced[team_next[t]] = True
            team_next[t] += T
            team_state[t] = "wait"
        elif kind == "issue":
            issued += 1
        else:
            completed[done % S] += 1
            done += 1
    return None


@pytest.mark.parametrize("T,S", [(2, 2), (2, 3), (2, 4), (3, 3), (3, 4)])
def test_teams_up_to_the_slot_count_never_alias(T, S):
    rng = random.Random(1000 * T + S)
    for _ in range(400):
        assert run(T, S, 48, rng) is None


@pytest.mark.parametrize("T,S", [(3, 2), (4, 3)])
def test_more_teams_than_slots_can_alias(T, S):
    rng = random.Random(7 * T + S)
    assert any(run(T, S, 48, rng) is not None for _ in range(400))
