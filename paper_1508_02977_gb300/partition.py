"""Subdomain partition of the pixel grid (Section 3.1).

The paper splits the image into px x py rectangular parts and prefers the
split with the largest area/perimeter ratio, area being the number of pixels
of a part and perimeter the number of pixels on its boundary, 2 (w + h) (the
worked example of Fig. ratio: a 48x48 grid in 12 parts gives 1.846 for 12x1,
3 for 6x2 and 3.428 for 4x3).  Here the same ratio is the prior of the tile
chooser: on the GPU a subdomain is a tile of T_x x T_y owned nodes handled by
one CTA, and a larger ratio means fewer overlap nodes per owned node.
"""
from __future__ import annotations


def part_ratio(W: int, H: int, px: int, py: int) -> float:
    """area / perimeter of one part when a W x H grid is cut into px x py
    equal parts (part size (W/px) x (H/py), perimeter 2 (w + h))."""
    w = W / px
    h = H / py
    return (w * h) / (2.0 * (w + h))


def splittings(nparts: int):
    """All (px, py) with px * py == nparts."""
    return [(px, nparts // px) for px in range(1, nparts + 1) if nparts % px == 0]


def best_split(W: int, H: int, nparts: int):
    """The (px, py) of largest area/perimeter ratio; ties go to the split
    with more parts along the longer side."""
    best = None
    for px, py in splittings(nparts):
        r = part_ratio(W, H, px, py)
        key = (round(r, 12), px if W >= H else py)
        if best is None or key > best[0]:
            best = (key, (px, py))
    return best[1]


def tiles_for(W: int, H: int, tile_x: int, tile_y: int):
    """Number of tiles along x and y for owned tiles of tile_x x tile_y
    nodes (the last tile of a row/column may be ragged)."""
    return (W + tile_x - 1) // tile_x, (H + tile_y - 1) // tile_y


def overlap_inflation(tile_x: int, tile_y: int, overlap: int) -> float:
    """Extended-tile nodes per owned node for an interior tile."""
    return (tile_x + 2 * overlap) * (tile_y + 2 * overlap) / float(tile_x * tile_y)
