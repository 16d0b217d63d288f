"""Thin-disk self-gravity on GB300 (sm_103a): the C-ABI library and its binding."""
