"""FP64 CPU oracle for the ProgOT hot path. Test infrastructure only: the CUDA
path never imports it (see progot_oracle's module notes)."""
from .progot_oracle import *  # noqa: F401,F403
