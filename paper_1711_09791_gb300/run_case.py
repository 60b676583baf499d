"""Run one configuration of the convolution on a synthetic image and print its
time: a command-line tool for measuring (or profiling) a single case.

    python -m paper_1711_09791_gb300.run_case --dtype bf16 --out bf16 --H 8192 --W 8192 --reps 20

Pixels are uniform in [0, 255) (seed 2), k is five seeded uniform values
normalised to sum 1; FP8 inputs use the scale 448/max.  Prints one JSON line
with the median kernel time (CUDA events) and the achieved algorithmic GB/s
(input read once plus output written once).

Options: --algo fused | two_pass | direct | reduce (one pyramid REDUCE step),
--layout planar | hwc, --tile TH,TW,STAGES (a compiled shape; TH and STAGES
for reduce), --ctas N (CTAs per SM; 0 = the planner's choice), --planes, --H,
--W, --reps, --warmup.
"""
from __future__ import annotations

import argparse
import json


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--dtype", default="f32", choices=["f32", "bf16", "f16", "fp8e4m3"])
    ap.add_argument("--out", default=None, help="output format (default: the input format)")
    ap.add_argument("--algo", default="fused", choices=["fused", "two_pass", "direct", "reduce"])
    ap.add_argument("--planes", type=int, default=3)
    ap.add_argument("--H", type=int, default=8192)
    ap.add_argument("--W", type=int, default=8192)
    ap.add_argument("--tile", default="", help="TH,TW,stages override")
    ap.add_argument("--layout", default="planar", choices=["planar", "hwc"])
    ap.add_argument("--ctas", type=int, default=0)
    ap.add_argument("--reps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    a = ap.parse_args()
    out_dtype = a.out or a.dtype

    import torch

    from . import sepconv5 as sc5
    from . import synth

    sc5.load()
    P, H, W = a.planes, a.H, a.W
    es, eo = sc5.DTYPE_BYTES[a.dtype], sc5.DTYPE_BYTES[out_dtype]
    pitch = -(-W * es // 16) * 16 // es
    opitch = -(-(W - 4) // 4) * 4
    g = torch.Generator(device="cuda").manual_seed(2)
    x = torch.rand((P, H, W), generator=g, device="cuda") * 255.0
    scale = 448.0 / float(x.max()) if a.dtype == "fp8e4m3" else 1.0
    tdt = {"f32": torch.float32, "bf16": torch.bfloat16, "f16": torch.float16, "fp8e4m3": torch.float8_e4m3fn}
    th = tw = st = 0
    if a.tile:
        th, tw, st = (int(v) for v in a.tile.split(","))
    if a.layout == "hwc":
        # the same pixels as RGB triples: value (p, y, x) at y * pitch + 3x + p
        pitch = -(-3 * W * es // 16) * 16 // es
        opitch = -(-3 * (W - 4) // 4) * 4
        A = torch.zeros((H, pitch), dtype=tdt[a.dtype], device="cuda")
        A[:, :3 * W] = (x * scale).permute(1, 2, 0).reshape(H, 3 * W).to(tdt[a.dtype])
        out = torch.empty((H - 4, opitch), dtype=tdt[out_dtype], device="cuda")
    else:
        A = torch.zeros((P, H, pitch), dtype=tdt[a.dtype], device="cuda")
        A[:, :, :W] = (x * scale).to(tdt[a.dtype])
        Ho, Wo = (sc5.reduce_dims(H, W) if a.algo == "reduce" else (H - 4, W - 4))
        opitch = -(-Wo * eo // 16) * 16 // eo if a.algo == "reduce" else opitch
        out = torch.empty((P, Ho, opitch), dtype=tdt[out_dtype], device="cuda")
    del x
    plan = sc5.Plan(P, H, W, pitch, opitch, a.dtype, out_dtype, "valid", a.algo, th, tw, st, a.ctas,
                    layout=a.layout)
    k = synth.kernel_normalised(2)
    out_scale = scale if out_dtype == "fp8e4m3" else 1.0
    stream = torch.cuda.current_stream()
    for _ in range(a.warmup):
        plan.run(A, out, k, scale, out_scale, stream=stream)
    times = []
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for _ in range(a.reps):
        e0.record(stream)
        plan.run(A, out, k, scale, out_scale, stream=stream)
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    times.sort()
    ms = times[len(times) // 2]
    Ho, Wo = (sc5.reduce_dims(H, W) if a.algo == "reduce" else (H - 4, W - 4))
    alg = P * H * W * es + P * Ho * Wo * eo
    if sc5.device_status(stream) != 0:
        raise SystemExit("a kernel reported a device error")
    plan.close()
    print(json.dumps({"dtype": a.dtype, "out": out_dtype, "algo": a.algo, "planes": P, "H": H, "W": W,
                      "layout": a.layout, "tile": a.tile or "default", "ms": round(ms, 5), "gbs": round(alg / ms / 1e6, 1),
                      "mpix_s": round(H * W / ms / 1e3, 1)}))


if __name__ == "__main__":
    main()
