"""Reader of the hand-worked scenario files in tests/golden/ (format in README.txt)."""
from __future__ import annotations

import os
import re

import numpy as np

GOLDEN_DIR = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")

_TERRAIN = {"": 0, "C": 2, "G": 3}
_DIRS = {"U": 0, "D": 1, "L": 2, "R": 3}
_CELL = re.compile(r"^(\d+)(?:@(\d))?([CG]?)$")


def parse_cell(tok: str):
    """-> (army, owner, terrain) of one cell token."""
    if tok == "M":
        return 0, -1, 1
    m = _CELL.match(tok)
    if not m:
        raise ValueError(f"bad cell token {tok!r}")
    army = int(m.group(1))
    owner = int(m.group(2)) if m.group(2) is not None else -1
    return army, owner, _TERRAIN[m.group(3)]


def parse_board(lines, H, W):
    army = np.zeros(H * W, np.int16)
    owner = np.zeros(H * W, np.int8)
    terrain = np.zeros(H * W, np.int8)
    for r, line in enumerate(lines):
        toks = line.split()
        assert len(toks) == W, f"row {r}: expected {W} cells, got {toks}"
        for c, tok in enumerate(toks):
            a, o, t = parse_cell(tok)
            army[r * W + c], owner[r * W + c], terrain[r * W + c] = a, o, t
    return army, owner, terrain


def parse_mode(tok: str):
    if tok == "1v1":
        return 0, 2
    if tok == "2v2":
        return 1, 4
    m = re.match(r"^ffa(\d)$", tok)
    if m:
        return 2, int(m.group(1))
    raise ValueError(tok)


def action_index(line: str, W: int) -> tuple[int, int]:
    """'p: row col DIR all|half' | 'p: pass' | 'p: raw k' -> (player, flat action)."""
    p, rest = line.split(":", 1)
    toks = rest.split()
    if toks[0] == "pass":
        return int(p), 0
    if toks[0] == "raw":
        return int(p), int(toks[1])
    r, c, d, kind = int(toks[0]), int(toks[1]), _DIRS[toks[2]], toks[3]
    k = (1 + d) if kind == "all" else (5 + d)
    return int(p), (r * W + c) * 9 + k


def _int_grid(lines):
    return np.array([[int(x) for x in ln.split()] for ln in lines], dtype=np.int64).reshape(-1)


def load(path: str) -> dict:
    raw = [ln.rstrip() for ln in open(path)]
    lines = [ln for ln in raw if ln.strip() and not ln.lstrip().startswith("#")]
    sc = {"name": os.path.basename(path), "alive": None, "max_turns": 0, "steps": []}
    i = 0
    H = W = None
    while i < len(lines):
        toks = lines[i].split()
        head = toks[0]
        if head == "mode":
            sc["mode"], sc["P"] = parse_mode(toks[1])
            i += 1
        elif head == "size":
            H, W = int(toks[1]), int(toks[2])
            sc["H"], sc["W"] = H, W
            i += 1
        elif head == "turn" and not sc["steps"]:
            sc["turn"] = int(toks[1])
            i += 1
        elif head == "alive" and not sc["steps"]:
            sc["alive"] = int(toks[1], 0)
            i += 1
        elif head == "max_turns":
            sc["max_turns"] = int(toks[1])
            i += 1
        elif head == "board":
            sc["board"] = parse_board(lines[i + 1:i + 1 + H], H, W)
            i += 1 + H
        elif head == "actions":
            acts = np.zeros(8, np.int32)
            i += 1
            for _ in range(sc["P"]):
                p, a = action_index(lines[i], W)
                acts[p] = a
                i += 1
            sc["steps"].append({"actions": acts, "checks": {}, "obs": {}, "scoreboard": None})
        elif head == "expect":
            step = sc["steps"][-1]
            step["board"] = parse_board(lines[i + 1:i + 1 + H], H, W)
            i += 1 + H
            while i < len(lines) and lines[i].split()[0] in ("turn", "alive", "invalid", "saturated", "done",
                                                              "reward"):
                t = lines[i].split()
                if t[0] == "reward":
                    step["checks"]["reward"] = [float(x) for x in t[1:]]
                elif t[0] == "alive":
                    step["checks"]["alive"] = int(t[1], 0)
                else:
                    step["checks"][t[0]] = int(t[1])
                i += 1
        elif head == "obs":
            step = sc["steps"][-1]
            p = int(toks[1])
            step["obs"][p] = {}
            i += 1
            while i < len(lines) and lines[i].split()[0] in ("vis", "terrain", "owner", "army", "mask"):
                name = lines[i].split()[0]
                step["obs"][p][name] = _int_grid(lines[i + 1:i + 1 + H])
                i += 1 + H
        elif head == "scoreboard":
            step = sc["steps"][-1]
            land = [int(x) for x in lines[i + 1].split()[1:]]
            army = [int(x) for x in lines[i + 2].split()[1:]]
            step["scoreboard"] = (land, army)
            i += 3
        else:
            raise ValueError(f"{path}: unknown line {lines[i]!r}")
    return sc


def all_scenarios():
    return sorted(os.path.join(GOLDEN_DIR, f) for f in os.listdir(GOLDEN_DIR) if f.endswith(".txt")
                  and f != "README.txt")
