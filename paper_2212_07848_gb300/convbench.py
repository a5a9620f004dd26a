"""Time one 3x3 convolution layer of the surrogate through the C ABI.

    python -m paper_2212_07848_gb300.convbench --nb 8 --h 128 --cin 64 --cout 128 --path 0

Runs the forward convolution (bias + ReLU), or with `--dgrad` the input
gradient of that layer, or with `--wgrad` its weight and bias gradients
(into a workspace), `--iters` times on random BF16 inputs after
`--warmup` calls and prints the mean time per call and the achieved TFLOP/s
(2 * 9 * cin * cout FLOP per output pixel).  `--path` selects the kernel (0
automatic, 1 mma.sync, 2 tcgen05 per tile, 3 persistent tcgen05) as in
`lb_nn_set_conv_path`.
"""
import argparse
import ctypes as C

from . import abi


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--nb", type=int, default=8)
    ap.add_argument("--h", type=int, default=128)
    ap.add_argument("--cin", type=int, default=64)
    ap.add_argument("--cout", type=int, default=128)
    ap.add_argument("--path", type=int, default=0)
    ap.add_argument("--warmup", type=int, default=2)
    ap.add_argument("--iters", type=int, default=3)
    ap.add_argument("--dgrad", action="store_true")
    ap.add_argument("--wgrad", action="store_true")
    a = ap.parse_args()
    import torch
    L = abi.load()
    p = lambda t: C.c_void_p(t.data_ptr())
    g = torch.Generator(device="cpu").manual_seed(0)
    x = torch.randn((a.nb, a.h, a.h, a.cin), generator=g).to(torch.bfloat16).cuda()
    w = (0.1 * torch.randn((9, a.cout, a.cin), generator=g)).to(torch.bfloat16).cuda()
    b = torch.zeros(a.cout, device="cuda")
    y = torch.empty((a.nb, a.h, a.h, a.cout), dtype=torch.bfloat16, device="cuda")
    if L.lb_nn_set_conv_path(a.path) != 0:
        raise SystemExit("bad --path")
    if a.wgrad:   # dL/dw [9][cout][cin] and dL/db [cout] from x and dL/dy
        L.lb_nn_conv3x3_wgrad.argtypes = [C.c_void_p] * 4 + [C.c_int] * 5 + [C.c_void_p,
                                                                            C.c_size_t,
                                                                            C.c_void_p]
        L.lb_nn_wgrad_workspace.argtypes = [C.c_int] * 5
        L.lb_nn_wgrad_workspace.restype = C.c_size_t
        dy = torch.randn((a.nb, a.h, a.h, a.cout), generator=g).to(torch.bfloat16).cuda()
        dw = torch.zeros((9, a.cout, a.cin), device="cuda")
        db = torch.zeros(a.cout, device="cuda")
        nbytes = L.lb_nn_wgrad_workspace(a.nb, a.h, a.h, a.cin, a.cout)
        ws = torch.empty(nbytes // 4, dtype=torch.float32, device="cuda")
        call = lambda: L.lb_nn_conv3x3_wgrad(p(x), p(dy), p(dw), p(db), a.nb, a.h, a.h, a.cin,
                                             a.cout, p(ws), nbytes, None)
    elif a.dgrad:   # dL/dx [..][cin] from dL/dy [..][cout] with the layer's weights
        dy = torch.randn((a.nb, a.h, a.h, a.cout), generator=g).to(torch.bfloat16).cuda()
        dx = torch.empty((a.nb, a.h, a.h, a.cin), dtype=torch.bfloat16, device="cuda")
        call = lambda: L.lb_nn_conv3x3(p(dy), p(w), None, p(dx), a.nb, a.h, a.h, a.cout, a.cin,
                                       0, 1, None)
    else:
        call = lambda: L.lb_nn_conv3x3(p(x), p(w), p(b), p(y), a.nb, a.h, a.h, a.cin, a.cout, 1,
                                       0, None)
    for _ in range(a.warmup):
        if call() != 0:
            raise SystemExit("the convolution call failed")
    s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s.record()
    for _ in range(a.iters):
        call()
    e.record()
    e.synchronize()
    if L.lb_nn_status() != 0:
        raise SystemExit("a tensor-core wait gave up")
    ms = s.elapsed_time(e) / a.iters
    flop = 2.0 * 9 * a.cin * a.cout * a.nb * a.h * a.h
    kind = "wgrad" if a.wgrad else ("dgrad" if a.dgrad else "fwd")
    print(f"{a.nb}x{a.h}^2 {a.cin}->{a.cout} {kind} path {a.path}: {ms * 1e3:.1f} us, "
          f"{flop / ms / 1e9:.1f} TFLOP/s")


if __name__ == "__main__":
    main()
