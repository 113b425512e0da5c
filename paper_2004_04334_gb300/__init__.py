"""GB300-native offloaded silicon-pixel local reconstruction (libhp)."""
