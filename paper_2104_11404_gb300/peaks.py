"""Measured FP64 and FP32 FMA rates of the GPU (the denominators of the
ALU-bound rooflines), from the library's probe kernel (lh_peak_probe).

    python -m paper_2104_11404_gb300.peaks            # prints one JSON line
    python -m paper_2104_11404_gb300.peaks --lanes    # FP64 time per warp instruction
                                                      # against its active lanes

Each precision: one untimed launch, then the best of `reps` launches timed
with CUDA events on the launching stream, iteration counts sized for
launches of roughly 20 ms.
"""
import json
import sys


def measure(stream=None, reps=5):
    import torch
    from . import build as libbuild
    from . import lagh
    libbuild.build()
    s = stream if stream is not None else torch.cuda.current_stream()
    sink = torch.zeros(8 * 1024, dtype=torch.float64, device="cuda")
    out = {}
    for name, fp64, iters in (("fp64_tflops", True, 6000), ("fp32_tflops", False, 200000)):
        lagh.lh_peak_probe(fp64, iters, sink, s.cuda_stream)
        best = None
        flops = 0.0
        for _ in range(reps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(s)
            flops = lagh.lh_peak_probe(fp64, iters, sink, s.cuda_stream)
            e1.record(s)
            e1.synchronize()
            ms = e0.elapsed_time(e1)
            best = ms if best is None or ms < best else best
        out[name] = flops / (best * 1e-3) / 1e12
        out[name.replace("tflops", "launch_ms")] = best
    return out


def lanes(stream=None, iters=6000, reps=3):
    """FP64 probe with the chains on 32, 16, 8, 4, 2 and 1 lanes of every warp:
    launch time and the pipe time of one warp-wide FMA instruction per SM."""
    import torch
    from . import build as libbuild
    from . import lagh
    libbuild.build()
    s = stream if stream is not None else torch.cuda.current_stream()
    sink = torch.zeros(8 * 1024, dtype=torch.float64, device="cuda")
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    out = []
    for n in (32, 16, 8, 4, 2, 1):
        lagh.lh_peak_probe_lanes(True, n, iters, sink, s.cuda_stream)
        best = None
        for _ in range(reps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(s)
            lagh.lh_peak_probe_lanes(True, n, iters, sink, s.cuda_stream)
            e1.record(s)
            e1.synchronize()
            ms = e0.elapsed_time(e1)
            best = ms if best is None or ms < best else best
        warp_instr_per_sm = 8 * 8 * 8 * iters  # blocks x warps x chains x iterations, per SM
        out.append({"lanes": n, "launch_ms": best,
                    "ns_per_warp_fma_per_sm": best * 1e6 / warp_instr_per_sm})
    return out


if __name__ == "__main__":
    import torch
    torch.cuda.set_device(0)
    if "--lanes" in sys.argv:
        print(json.dumps({"fp64_lanes": lanes(), "device": torch.cuda.get_device_name(0)}))
        sys.exit(0)
    res = measure()
    res["device"] = torch.cuda.get_device_name(0)
    print(json.dumps(res))
    sys.exit(0)
