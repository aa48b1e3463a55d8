"""FP64 CPU oracle of the LoRADS hot path.  TEST INFRASTRUCTURE: used only by
tests/, __graft_entry__.smoke() and bench.py's CPU-baseline / reference legs."""
