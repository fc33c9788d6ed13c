"""Host-side checks of the 2D tile kernels' index arithmetic for every mesh
size up to a few hundred node lines (the GPU tests cover a handful of sizes).

This mirrors the tiling of cg_pass2d_kernel and cg_apply2d_kernel: 16-wide
tiles of node lines, a single remaining line joining the last tile (17
wide), and for the fused mass apply the elements that touch a tile's nodes,
whose count is bounded by the kernel's shared-memory patch."""
import pytest

TS, TM = 16, 17


def tiles(n):
    t = (n + TS - 1) // TS
    return t - 1 if (n % TS == 1 and t > 1) else t


def tile_extent(n, i):
    nt = tiles(n)
    x0 = i * TS
    return x0, (n - x0 if i == nt - 1 else TS)


def node_elements(x, k, nel):
    """Elements along one direction that contain node x (increasing)."""
    q, r = divmod(x, k)
    if r:
        return [q]
    return ([q - 1] if q > 0 else []) + ([q] if q < nel else [])


@pytest.mark.parametrize("n", range(2, 400))
def test_tiles_cover_every_node_line_once(n):
    seen = []
    for i in range(tiles(n)):
        x0, w = tile_extent(n, i)
        assert 1 <= w <= TM
        seen.extend(range(x0, x0 + w))
    assert seen == list(range(n))


@pytest.mark.parametrize("k", [1, 2, 3])
def test_apply_patch_holds_every_touching_element(k):
    ne1 = (TS + 1 + k - 1) // k + 1          # elements touching 17 node lines
    npn = k * ne1 + 1                          # their node lines
    for nel in range(1, 140):
        n = k * nel + 1
        for i in range(tiles(n)):
            x0, w = tile_extent(n, i)
            ex0 = (x0 - 1) // k if x0 > 0 else 0
            ex1 = min(nel - 1, (x0 + w - 1) // k)
            nex = ex1 - ex0 + 1
            assert 1 <= nex <= ne1 and k * nex + 1 <= npn
            for x in range(x0, x0 + w):
                els = node_elements(x, k, nel)
                assert els and all(ex0 <= e <= ex1 for e in els), (k, nel, i, x)
                # the node's patch column lies inside the staged patch
                assert 0 <= x - k * ex0 < k * nex + 1
