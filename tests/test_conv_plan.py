"""Host-side checks of the two convolution plans (no GPU): for every layer shape the
denoiser and the convolution tests launch, the plan the library would use keeps every
bulk copy, every tensor-core operand read and every accumulator inside its buffer.

The invariants restate the kernels' addressing (brick convolution: the producer's six
brick runs per 16-channel chunk, the A windows of the 27 taps per M tile, the weight
chunk, the accumulators and the fold's exchange buffer; weight gradient: the dy rows,
the input brick and the tap accumulators), so that a change of the cost model cannot
pick a layout that would read or write outside shared or tensor memory on the GPU."""
import itertools

import pytest

import paper_2511_03115_gb300 as S

SMEM_CAP = 227 * 1024
HEADER = 1024  # barriers, tensor-memory slot and abort flag before the stages
STAGES = 2

# The denoiser's eleven convolutions: (input channels, output channels, pooling level).
LAYERS = [(16, 32, 0), (32, 32, 0), (32, 64, 1), (64, 64, 1), (64, 128, 2), (128, 128, 2),
          (192, 64, 1), (64, 64, 1), (96, 32, 0), (32, 32, 0), (32, 16, 0)]
# Grids (D, H, W) the denoiser is created on: the 128 x 128 x 192 workload, the GPU
# tests' small volumes and the smoke check's.
GRIDS = [(192, 128, 128), (16, 16, 32), (8, 16, 32), (8, 16, 16)]
# The convolution tests' shapes: (Cin, Cout, (D, H, W)).
CONV_TESTS = [(16, 32, (4, 8, 8)), (32, 64, (3, 8, 16)), (96, 32, (2, 8, 8)), (192, 64, (2, 4, 16)),
              (64, 128, (4, 4, 8)), (32, 32, (3, 5, 128)), (32, 96, (2, 9, 64)), (32, 16, (4, 7, 32)),
              (16, 32, (2, 3, 256)), (32, 96, (2, 4, 128)), (16, 32, (2, 6, 128)), (32, 16, (3, 4, 128))]


def _forward_shapes():
    out = set()
    for D, H, W in GRIDS:
        for cin, cout, lv in LAYERS:
            d, h, w = D >> lv, H >> lv, W >> lv
            out.add((d, h, w, cin, cout))   # forward
            out.add((d, h, w, cout, cin))   # data gradient: forward with flipped weights
    for cin, cout, (D, H, W) in CONV_TESTS:
        out.add((D, H, W, cin, cout))
        out.add((D, H, W, cout, cin))
    return sorted(s for s in out if s[3] <= 192)  # the data gradient of the input layer is not formed


def _wgrad_shapes():
    out = set()
    for D, H, W in GRIDS:
        for cin, cout, lv in LAYERS:
            out.add((D >> lv, H >> lv, W >> lv, cin, cout))
    for cin, cout, (D, H, W) in CONV_TESTS:
        if cout <= 128:
            out.add((D, H, W, cin, cout))
    return sorted(out)


@pytest.mark.parametrize("D,H,W,Cin,Cout", _forward_shapes())
@pytest.mark.parametrize("batch", [1, 2])
def test_brick_plan_stays_inside_its_buffers(D, H, W, Cin, Cout, batch):
    b = S.conv3d_plan(batch, D, H, W, Cin, Cout)
    Ty, tiles, P, Yb, Cp, plane = b["Ty"], b["tiles"], b["P"], b["Yb"], b["Cp"], b["plane"]
    nchunk = Cin // 16
    w_bytes = 27 * Cp * 32  # one chunk's weights: 27 taps x Cp x 16 BF16
    assert P == W + 2 and Yb == Ty + 2 and Cout % Cp == 0 and b["nsplit"] == Cout // Cp and Cp % 16 == 0
    assert b["nyb"] == -(-H // Ty) and b["items"] == batch * b["nsplit"] * b["nyb"] * D
    rowtile = W % 128 == 0
    assert b["rowtile"] == int(rowtile)
    tpr = W // 128
    if rowtile:
        assert tiles == Ty * tpr
    else:
        assert tiles * 128 >= Ty * P  # flat tiles cover the item's rows with their padding columns
    if b["fold"]:
        assert rowtile and tpr == 1 and tiles <= 4 and 3 * Cp <= 256
    else:
        assert tiles <= 8
    # tensor memory: nacc accumulators of tiles x Cp (x 3 folded) columns
    acc_cols = tiles * Cp * (3 if b["fold"] else 1)
    assert b["tcols"] in (32, 64, 128, 256, 512) and b["nacc"] in (1, 2)
    assert b["nacc"] * acc_cols <= b["tcols"]
    # a stage: 128 bytes, then the chunk's two 8-channel planes of three brick runs each
    slot = Yb * P * 16
    assert plane >= 3 * slot and plane % 128 == 0 and plane < 1 << 18
    assert 128 + plane + 3 * slot <= b["w_off"]
    # the A windows of all taps and tiles, in positions from the stage's brick start
    lo, hi = None, None
    for (dz, dy, dx), m in itertools.product(itertools.product((-1, 0, 1), repeat=3), range(tiles)):
        base = (Yb + 1) * P + 1 + (m // tpr) * P + (m % tpr) * 128 if rowtile else (Yb + 1) * P + 128 * m
        start = base + (dz * Yb + dy) * P + dx
        lo = start if lo is None else min(lo, start)
        hi = start + 127 if hi is None else max(hi, start + 127)
    # flat tiles start one position before the brick (inside the stage's first 128 bytes;
    # that row is a padding column the epilogue drops)
    assert 128 + 16 * lo >= 0
    if rowtile:
        assert lo >= 0 and hi < 3 * Yb * P  # inside the three staged plane runs
    # the second K half reads `plane` bytes further; both end before the weights
    assert 128 + plane + 16 * (hi + 1) <= b["w_off"]
    if b["wres"]:
        assert b["stage"] == b["w_off"]
        assert b["xch"] == HEADER + STAGES * b["stage"] + nchunk * w_bytes
    else:
        assert b["w_off"] + w_bytes <= b["stage"]
        assert b["xch"] == HEADER + STAGES * b["stage"]
    assert b["stage"] % 128 == 0 and b["w_off"] % 128 == 0
    # the fold's exchange buffer: two groups x two tiles x two edges x 4 quarters x Cp floats
    assert b["smem"] == b["xch"] + (128 * Cp if b["fold"] else 0)
    assert b["smem"] <= SMEM_CAP
    # global reads: rows y0 - 1 .. y0 - 1 + rows - 1 of the padded plane, rows = min(Yb, H + 2 - y0),
    # cover rows y - 1 .. y + 1 of every output row y < H of the item
    for y0 in range(0, H, Ty):
        rows = min(Yb, H + 2 - y0)
        assert y0 - 1 + rows - 1 <= H
        for y in range(y0, min(y0 + Ty, H)):
            assert (y - y0) + 2 < rows


@pytest.mark.parametrize("D,H,W,Cin,Cout", _wgrad_shapes())
@pytest.mark.parametrize("sms", [152, 132])
def test_wgrad_plan_stays_inside_its_buffers(D, H, W, Cin, Cout, sms):
    b = S.conv3d_wgrad_plan(1, D, H, W, Cin, Cout, sms=sms)
    Ty, P, Yb, Nc = b["Ty"], b["P"], b["Yb"], b["Nc"]
    assert P == W + 2 and Yb == Ty + 2 and H % Ty == 0 and b["nyb"] == H // Ty and b["items"] == b["nyb"] * D
    assert Nc in (16, 32) and Cin % Nc == 0
    # each pass's tap accumulators fit the 512 tensor-memory columns; the groups cover 27 taps
    assert b["ntap"] * Nc <= 512 and b["ngroups"] * b["ntap"] >= 27 > (b["ngroups"] - 1) * b["ntap"]
    # dy rows: Ty P positions per 8-channel plane, K steps of 16 positions
    assert b["kst"] == -(-Ty * P // 16) and b["plane_dy"] == 256 * b["kst"]
    assert b["plane_dy"] < 1 << 18 and b["plane_x"] < 1 << 18
    # the input brick starts after the dy planes with room for the read one position before it
    assert b["x_off"] >= (Cout // 8) * b["plane_dy"] + 16 and b["x_off"] % 128 == 0
    assert b["plane_x"] >= 3 * Yb * P * 16 and b["plane_x"] % 128 == 0
    # B windows: positions (Yb + 1) P + tap offset + 16 ks .. + 15, at most 16 past the brick
    top = (Yb + 1) * P + ((Yb + 1) * P + 1) + 16 * (b["kst"] - 1) + 15
    assert top < 3 * Yb * P + 16
    assert b["x_off"] + (Nc // 8 - 1) * b["plane_x"] + 16 * (top + 1) <= b["stage"]
    # the A operand (M = 128 rows: output channels padded) stays inside the stage
    assert b["stage"] >= 16 * b["plane_dy"] and b["stage"] % 128 == 0
    assert b["smem"] == HEADER + STAGES * b["stage"] <= SMEM_CAP
    # all passes in one wave on the SMs, each with at least one CTA
    passes = (Cin // Nc) * b["ngroups"]
    assert 1 <= b["G"] <= b["items"]
    assert b["G"] * passes <= sms or b["G"] == 1


def test_plans_reject_shapes_the_kernels_do_not_take():
    for args in [(1, 8, 8, 300, 16, 16), (1, 8, 8, 8, 8, 16), (1, 8, 8, 8, 16, 8), (1, 8, 8, 8, 208, 16),
                 (0, 8, 8, 8, 16, 16)]:
        with pytest.raises(S.SdeError):
            S.conv3d_plan(*args)
    with pytest.raises(S.SdeError):
        S.conv3d_wgrad_plan(1, 8, 8, 8, 16, 256)  # the weight gradient takes Cout <= 128
    with pytest.raises(S.SdeError):
        S.conv3d_wgrad_plan(1, 8, 8, 8, 16, 16, sms=0)
